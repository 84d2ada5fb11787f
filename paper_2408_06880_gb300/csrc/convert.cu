// convert.cu -- change of the storage format of a domain's populations.
//
// The populations are stored shifted (g_i = f_i - w_i, the paper's
// zero-centred storage, Sec. 4) as FP32, or as FP16 / BF16 holding g_i * 2^s
// with a per-domain power-of-two scale s.  A conversion maps every stored
// value v (format A, scale s_a) to pack_B(raw_A(v) * 2^(s_b - s_a)):
//   - FP16/BF16 -> FP32 and a rescale within FP16/BF16 by a power of two are
//     exact (the FP32 product of a 16-bit value and a power of two is exact,
//     and so is its rounding back to the 16-bit format while the result is a
//     normal number and in range; values in the subnormal range round);
//   - FP32 -> FP16/BF16 rounds to nearest even, as every store of the
//     stepping kernels does.
// The conversion is element-wise over the whole Q x S array (both fields of
// the pull layout), so it holds at either AA parity: every slot keeps its
// meaning.  Before converting, the largest |raw| is found on the device and a
// conversion that would overflow the target format is refused.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace slbm {

template <int SS, int DS>
__global__ void convert_kernel(const typename Store<SS>::T *src, typename Store<DS>::T *dst, int64_t n, float mul) {
    // src may equal dst (same element size): each thread reads its element
    // before writing it
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
        dst[j] = Store<DS>::pack(Store<SS>::raw(src[j]) * mul);
}

// Largest |raw value| of n stored values, as the bits of a non-negative float
// (their integer order is the float order; a NaN's bits exceed infinity's),
// combined into *out with atomicMax (the result does not depend on order).
template <int ST>
__global__ void absmax_kernel(const typename Store<ST>::T *x, int64_t n, unsigned *out) {
    unsigned m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const unsigned b = __float_as_uint(fabsf(Store<ST>::raw(x[j])));
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

namespace {

constexpr int CONV_THREADS = 256;

unsigned grid_for(int64_t n) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + CONV_THREADS - 1) / CONV_THREADS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(sms, 1) * 8));
}

template <int SS>
cudaError_t launch_absmax(const void *x, int64_t n, unsigned *out, cudaStream_t st) {
    absmax_kernel<SS><<<grid_for(n), CONV_THREADS, 0, st>>>((const typename Store<SS>::T *)x, n, out);
    return cudaGetLastError();
}

cudaError_t absmax_any(int storage, const void *x, int64_t n, unsigned *out, cudaStream_t st) {
    switch (storage) {
        case SLBM_FP32: return launch_absmax<ST_F32>(x, n, out, st);
        case SLBM_FP16: return launch_absmax<ST_F16>(x, n, out, st);
        default: return launch_absmax<ST_BF16>(x, n, out, st);
    }
}

template <int SS, int DS>
cudaError_t launch_convert(const void *src, void *dst, int64_t n, float mul, cudaStream_t st) {
    convert_kernel<SS, DS><<<grid_for(n), CONV_THREADS, 0, st>>>((const typename Store<SS>::T *)src,
                                                                  (typename Store<DS>::T *)dst, n, mul);
    return cudaGetLastError();
}

template <int SS>
cudaError_t convert_from(int ds, const void *src, void *dst, int64_t n, float mul, cudaStream_t st) {
    switch (ds) {
        case SLBM_FP32: return launch_convert<SS, ST_F32>(src, dst, n, mul, st);
        case SLBM_FP16: return launch_convert<SS, ST_F16>(src, dst, n, mul, st);
        default: return launch_convert<SS, ST_BF16>(src, dst, n, mul, st);
    }
}

cudaError_t convert_any(int ss, int ds, const void *src, void *dst, int64_t n, float mul, cudaStream_t st) {
    switch (ss) {
        case SLBM_FP32: return convert_from<ST_F32>(ds, src, dst, n, mul, st);
        case SLBM_FP16: return convert_from<ST_F16>(ds, src, dst, n, mul, st);
        default: return convert_from<ST_BF16>(ds, src, dst, n, mul, st);
    }
}

}  // namespace

int convert_storage(Ctx &cx, Domain &d, int storage, int scale_exp) {
    const int new_s = storage == SLBM_FP32 ? 0 : scale_exp;
    const int old_s = d.storage == SLBM_FP32 ? 0 : d.scale_exp;
    const int64_t n = (int64_t)d.q * d.S;
    DevBuf *fields[2] = {&d.pdf, d.pull() ? &d.pdf2 : nullptr};
    if (n > 0) {
        // largest stored magnitude of the current state, in raw units
        unsigned *m = (unsigned *)d.red_out.p;
        if (cx.check(cudaMemsetAsync(m, 0, sizeof(unsigned), d.stream), "memset"))
            return -1;
        for (DevBuf *f : fields)
            if (f && cx.check(absmax_any(d.storage, f->p, n, m, d.stream), "absmax")) return -1;
        unsigned bits = 0;
        if (cx.check(cudaMemcpyAsync(&bits, m, sizeof(unsigned), cudaMemcpyDeviceToHost, d.stream), "absmax D2H") ||
            cx.check(cudaStreamSynchronize(d.stream), "absmax sync"))
            return -1;
        float amax;
        std::memcpy(&amax, &bits, sizeof(float));
        if (!std::isfinite(amax)) {
            cx.fail(SLBM_EDIVERGED, "the stored populations are not finite");
            return -1;
        }
        const double target = std::ldexp((double)amax, new_s - old_s);
        const double limit = storage == SLBM_FP16 ? 65504.0 : (storage == SLBM_BF16 ? 3.38e38 : 3.4e38);
        if (target >= limit) {
            const std::string m = "the converted populations would overflow the target format (largest |g| * 2^s = " +
                                  std::to_string(target) + ")";
            cx.fail(SLBM_EINVAL, m.c_str());
            return -1;
        }
        const float mul = std::ldexp(1.0f, new_s - old_s);
        const int new_b = storage == SLBM_FP32 ? 4 : 2;
        if (new_b == d.bytes_per_pdf()) {              // in place, element by element
            for (DevBuf *f : fields)
                if (f && cx.check(convert_any(d.storage, storage, f->p, f->p, n, mul, d.stream), "convert")) return -1;
        } else {                                       // new arrays first: a failure leaves the domain as it was
            DevBuf nb[2];
            for (int j = 0; j < 2; ++j) {
                if (!fields[j]) continue;
                if (cx.alloc(nb[j], n * new_b) ||
                    cx.check(convert_any(d.storage, storage, fields[j]->p, nb[j].p, n, mul, d.stream), "convert")) {
                    cudaStreamSynchronize(d.stream);
                    cx.release(nb[0]);
                    cx.release(nb[1]);
                    return -1;
                }
            }
            if (cx.check(cudaStreamSynchronize(d.stream), "convert sync")) {
                cx.release(nb[0]);
                cx.release(nb[1]);
                return -1;
            }
            for (int j = 0; j < 2; ++j) {
                if (!fields[j]) continue;
                cx.release(*fields[j]);
                *fields[j] = nb[j];
            }
        }
        if (cx.check(cudaStreamSynchronize(d.stream), "convert sync")) return -1;
    }
    d.storage = storage;
    d.scale_exp = new_s;
    return 0;
}

}  // namespace slbm
