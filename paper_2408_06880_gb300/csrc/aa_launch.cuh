// aa_launch.cuh -- host dispatch of the AA kernels for one stencil size.
#pragma once

#include <mutex>
#include <tuple>

#include "aa_kernels.cuh"
#include "aa_window.cuh"
#include "brick.cuh"
#include "internal.h"

namespace slbm {

// Link tables of a domain for the even kernels that apply the link maps.
static EvenLinks even_links_of(const Domain &d) {
    return EvenLinks{(const int32_t *)d.ltile.p, (const int32_t *)d.link_cell.p, (const int32_t *)d.link_dir.p,
                     (const LinkMap *)d.link_map.p};
}

// Persistent grid: SMs x resident CTAs of this kernel at this block size and
// dynamic shared memory on the current device (looked up once each).
template <class K>
static unsigned persistent_grid(K kernel, int threads, int64_t tiles, size_t smem = 0) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    int slots;
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto key = std::make_tuple(dev, (const void *)kernel, threads, smem);
        auto it = cache.find(key);
        if (it == cache.end()) {
            int sms = 1, ctas = 1;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, kernel, threads, smem);
            it = cache.emplace(key, std::max(sms, 1) * std::max(ctas, 1)).first;
        }
        slots = it->second;
    }
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, slots));
}

// PACK (even step only): 2 cells per thread, collided in pairs.
template <int Q, int ST, int TILE, int NSTAGE, bool PACK = false>
static cudaError_t launch_staged(const Domain &d, int parity, cudaStream_t st) {
    using T = typename Store<ST>::T;
    T *pdf = reinterpret_cast<T *>(d.pdf.p);
    const int32_t S = (int32_t)d.S, nf = (int32_t)d.n_fluid;
    const CollideParams p = d.collide_params();
    int32_t *err = reinterpret_cast<int32_t *>(d.err.p);
    const int64_t tiles = S / TILE;
    if (parity == 0) {
        const bool bc = d.n_links > 0;
        const EvenLinks lk = bc ? even_links_of(d) : EvenLinks{};
        if constexpr (ST == ST_F16 || PACK) {    // 2 cells per thread (FP16: paired conversions)
            auto k = bc ? aa_even_staged_kernel<Q, ST, TILE, NSTAGE, 2, PACK, true>
                        : aa_even_staged_kernel<Q, ST, TILE, NSTAGE, 2, PACK, false>;
            k<<<persistent_grid(k, TILE / 2, tiles), TILE / 2, 0, st>>>(pdf, S, nf, p, err, lk);
        } else {
            auto k = bc ? aa_even_staged_kernel<Q, ST, TILE, NSTAGE, 1, false, true>
                        : aa_even_staged_kernel<Q, ST, TILE, NSTAGE, 1, false, false>;
            k<<<persistent_grid(k, TILE, tiles), TILE, 0, st>>>(pdf, S, nf, p, err, lk);
        }
    } else if constexpr (!PACK) {
        const int32_t *P = reinterpret_cast<const int32_t *>(d.P.p);
        const LinkMap *maps = reinterpret_cast<const LinkMap *>(d.link_map.p);
        if (d.n_links > 0) {
            auto k = aa_odd_staged_kernel<Q, ST, true, TILE, NSTAGE>;
            k<<<persistent_grid(k, TILE, tiles), TILE, 0, st>>>(pdf, P, S, nf, maps, p, err);
        } else {
            auto k = aa_odd_staged_kernel<Q, ST, false, TILE, NSTAGE>;
            k<<<persistent_grid(k, TILE, tiles), TILE, 0, st>>>(pdf, P, S, nf, maps, p, err);
        }
    }
    return cudaGetLastError();
}

// Odd step from bulk-staged tiles and neighbour windows (launch variant 6),
// NSTAGE stages in dynamic shared memory.
template <int Q, int ST, bool BC, int NSTAGE>
static cudaError_t launch_window_n(const Domain &d, cudaStream_t st) {
    using T = typename Store<ST>::T;
    auto k = aa_odd_window_kernel<Q, ST, BC, NSTAGE>;
    const size_t smem = window_smem_bytes<Q, ST>(NSTAGE);
    {   // the dynamic shared memory above 48 KB, set once per device before the occupancy query
        static std::mutex mu;
        static std::map<int, bool> done;
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lock(mu);
        if (!done[dev]) {
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    const int32_t S = (int32_t)d.S;
    k<<<persistent_grid(k, WIN_TILE + 32, S / WIN_TILE, smem), WIN_TILE + 32, smem, st>>>(
        reinterpret_cast<T *>(d.pdf.p), reinterpret_cast<const int32_t *>(d.P.p), S, (int32_t)d.n_fluid,
        reinterpret_cast<const WinSpan *>(d.win_tab.p), reinterpret_cast<const uint16_t *>(d.win_code.p),
        reinterpret_cast<const LinkMap *>(d.link_map.p),
        d.collide_params(), reinterpret_cast<int32_t *>(d.err.p));
    return cudaGetLastError();
}

template <int Q, int ST, bool BC>
static cudaError_t launch_window(const Domain &d, int nstage, cudaStream_t st) {
    switch (nstage) {
        case 2: return launch_window_n<Q, ST, BC, 2>(d, st);
        case 3: return launch_window_n<Q, ST, BC, 3>(d, st);
        case 4: return launch_window_n<Q, ST, BC, 4>(d, st);
        default: return cudaErrorInvalidValue;
    }
}

// Boundary fix-up launches around a pool's even step for a member with links
// (every even kernel of a domain of its own applies the link maps itself).
template <int Q, int ST>
cudaError_t launch_bc_pre(const Domain &d, cudaStream_t st) {
    const int32_t nb = (int32_t)d.n_bcells;
    if (nb == 0) return cudaSuccess;
    bc_pre_kernel<Q, ST><<<(nb + 127) / 128, 128, 0, st>>>(reinterpret_cast<const typename Store<ST>::T *>(d.pdf.p),
                                                           (int32_t)d.S, (const int32_t *)d.bcell.p, nb,
                                                           d.collide_params(), (float *)d.bc_ubuf.p);
    return cudaGetLastError();
}

template <int Q, int ST>
cudaError_t launch_bc_post(const Domain &d, cudaStream_t st) {
    const int32_t nb = (int32_t)d.n_bcells;
    if (nb == 0) return cudaSuccess;
    bc_post_kernel<ST><<<(nb + 127) / 128, 128, 0, st>>>(
        reinterpret_cast<typename Store<ST>::T *>(d.pdf.p), (int32_t)d.S, (const int32_t *)d.bcell.p,
        (const int32_t *)d.bfirst.p, nb, (const int32_t *)d.link_dir.p, (const LinkMap *)d.link_map.p,
        (const float *)d.bc_ubuf.p, d.collide_params().scale);
    return cudaGetLastError();
}

// The plain even kernel, `threads` x CPT cells a block, with the link maps
// folded in when the domain has inlet/outlet links.
template <int Q, int ST, int CPT, int OP = OP_TRT, bool PACK = false>
static cudaError_t launch_even_plain(const Domain &d, int threads, cudaStream_t st) {
    using T = typename Store<ST>::T;
    T *pdf = reinterpret_cast<T *>(d.pdf.p);
    const int32_t S = (int32_t)d.S, nf = (int32_t)d.n_fluid;
    const CollideParams p = d.collide_params();
    const dim3 grid((unsigned)((nf + threads * CPT - 1) / (threads * CPT)));
    if (d.n_bcells > 0)
        aa_even_kernel<Q, ST, CPT, OP, PACK, true><<<grid, threads, 3 * threads * CPT * sizeof(float), st>>>(
            pdf, S, nf, p, even_links_of(d));
    else
        aa_even_kernel<Q, ST, CPT, OP, PACK, false><<<grid, threads, 0, st>>>(pdf, S, nf, p);
    return cudaGetLastError();
}

// MRT (D3Q19), central-moment and cumulant (D3Q27) domains: the plain even
// kernel (1 or 2 cells per thread; MRT variant 2: the 2 cells collided in
// pairs; variant 5: 128 x 1 held to five resident blocks) and the odd kernel
// (1 or 2 cells, L2 index prefetch unless variant 0; variant 3: slots re-read
// before the scatter, no links; variant 5: 128 x 1 held to five resident
// blocks; checked mode), with the operator's collision.
template <int Q, int ST, int OP>
static cudaError_t launch_moment_op(const Domain &d, int parity, cudaStream_t st) {
    using T = typename Store<ST>::T;
    T *pdf = reinterpret_cast<T *>(d.pdf.p);
    const int32_t S = (int32_t)d.S, nf = (int32_t)d.n_fluid;
    const LaunchShape sh = d.shape[parity];
    const CollideParams p = d.collide_params();
    auto grid = [&](int cells) { return dim3((unsigned)((nf + sh.threads * cells - 1) / (sh.threads * cells))); };
    if (parity == 0) {
        if (sh.variant == 5) {                 // register-bounded, 128 x 1
            const dim3 g5((unsigned)((nf + 127) / 128));
            if (d.n_bcells > 0)
                aa_even_kernel_b5<Q, ST, OP, true><<<g5, 128, 3 * 128 * sizeof(float), st>>>(pdf, S, nf, p,
                                                                                            even_links_of(d));
            else
                aa_even_kernel_b5<Q, ST, OP, false><<<g5, 128, 0, st>>>(pdf, S, nf, p, EvenLinks{});
            return cudaGetLastError();
        }
        if (sh.cells == 1) return launch_even_plain<Q, ST, 1, OP>(d, sh.threads, st);
        if constexpr (OP == OP_MRT) {
            if (sh.variant == 2) return launch_even_plain<Q, ST, 2, OP, true>(d, sh.threads, st);
        }
        return launch_even_plain<Q, ST, 2, OP>(d, sh.threads, st);
    }
    const int32_t *P = reinterpret_cast<const int32_t *>(d.P.p);
    const LinkMap *maps = reinterpret_cast<const LinkMap *>(d.link_map.p);
    const int32_t nl = (int32_t)d.n_links;
    int32_t *err = reinterpret_cast<int32_t *>(d.err.p);
    const bool bc = nl > 0;
    if (d.checked) {
        auto kc = bc ? aa_odd_kernel<Q, ST, 1, true, true, false, false, OP>
                     : aa_odd_kernel<Q, ST, 1, false, true, false, false, OP>;
        kc<<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, 0, nullptr, nullptr);
        return cudaGetLastError();
    }
    if (sh.variant == 5) {                     // register-bounded, 128 x 1, L2 index prefetch
        auto kb = bc ? aa_odd_kernel_b5<Q, ST, OP, true> : aa_odd_kernel_b5<Q, ST, OP, false>;
        const int32_t pfb = (int32_t)persistent_grid(kb, 128, INT32_MAX);
        kb<<<(unsigned)((nf + 127) / 128), 128, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pfb);
        return cudaGetLastError();
    }
    if (sh.variant == 3 && !bc) {              // slots re-read before the scatter, L2 index prefetch
        auto kr = aa_odd_kernel<Q, ST, 1, false, false, true, false, OP>;
        const int32_t pfr = (int32_t)persistent_grid(kr, sh.threads, INT32_MAX);
        kr<<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pfr, nullptr, nullptr);
        return cudaGetLastError();
    }
    const int cells = sh.cells == 2 ? 2 : 1;
    auto k = cells == 1 ? (bc ? aa_odd_kernel<Q, ST, 1, true, false, false, false, OP>
                              : aa_odd_kernel<Q, ST, 1, false, false, false, false, OP>)
                        : (bc ? aa_odd_kernel<Q, ST, 2, true, false, false, false, OP>
                              : aa_odd_kernel<Q, ST, 2, false, false, false, false, OP>);
    const int32_t pf = sh.variant == 2 ? (int32_t)persistent_grid(k, sh.threads, INT32_MAX) : 0;
    k<<<grid(cells), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pf, nullptr, nullptr);
    return cudaGetLastError();
}

// Even step with the paired collision: variant 3 bulk-staged (tile `threads`
// cells, `cells` stages; FP32/FP16), variant 2 -- and variant 3 in checked
// mode -- the plain kernel with `cells` (2 or 4) cells per thread.
template <int Q, int ST>
static cudaError_t launch_even_packed(const Domain &d, const LaunchShape &sh, cudaStream_t st) {
    if constexpr (ST != ST_BF16) {
        if (sh.variant == 3 && !d.checked) {
            switch (sh.threads * 10 + sh.cells) {
                case 642: return launch_staged<Q, ST, 64, 2, true>(d, 0, st);
                case 644: return launch_staged<Q, ST, 64, 4, true>(d, 0, st);
                case 1282: return launch_staged<Q, ST, 128, 2, true>(d, 0, st);
                case 1284: return launch_staged<Q, ST, 128, 4, true>(d, 0, st);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    switch (sh.cells) {
        case 2: return launch_even_plain<Q, ST, 2, OP_TRT, true>(d, sh.threads, st);
        case 4: return launch_even_plain<Q, ST, 4, OP_TRT, true>(d, sh.threads, st);
        default: return cudaErrorInvalidValue;
    }
}

// One AA step of a domain with stencil Q and storage ST (instantiated per
// stencil and storage in aa_q<Q>_<storage>.cu).
template <int Q, int ST>
cudaError_t launch_aa_storage(const Domain &d, int parity, cudaStream_t st) {
    using T = typename Store<ST>::T;
    T *pdf = reinterpret_cast<T *>(d.pdf.p);
    const int32_t S = (int32_t)d.S, nf = (int32_t)d.n_fluid;
    if (nf == 0) return cudaSuccess;
    if constexpr (Q == 19) {
        if (d.op == SLBM_MRT) return launch_moment_op<19, ST, OP_MRT>(d, parity, st);
    }
    if constexpr (Q == 27) {
        if (d.op == SLBM_CM) return launch_moment_op<27, ST, OP_CM>(d, parity, st);
        if (d.op == SLBM_CUMULANT) return launch_moment_op<27, ST, OP_CUM>(d, parity, st);
    }
    const LaunchShape sh = d.shape[parity];
    if (parity == 0 && sh.variant >= 2) return launch_even_packed<Q, ST>(d, sh, st);
    if constexpr (ST != ST_BF16) {
        if (sh.variant == 1 && !d.checked) {
            switch (sh.threads * 10 + sh.cells) {
                case 642: return launch_staged<Q, ST, 64, 2>(d, parity, st);
                case 644: return launch_staged<Q, ST, 64, 4>(d, parity, st);
                case 1282: return launch_staged<Q, ST, 128, 2>(d, parity, st);
                case 1284: return launch_staged<Q, ST, 128, 4>(d, parity, st);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    const CollideParams p = d.collide_params();
    auto grid = [&](int cells) { return dim3((unsigned)((nf + sh.threads * cells - 1) / (sh.threads * cells))); };
    if (parity == 0) {
        switch (sh.cells) {
            case 1: return launch_even_plain<Q, ST, 1>(d, sh.threads, st);
            case 2: return launch_even_plain<Q, ST, 2>(d, sh.threads, st);
            case 4: return launch_even_plain<Q, ST, 4>(d, sh.threads, st);
            default: return cudaErrorInvalidValue;
        }
    }
    const int32_t *P = reinterpret_cast<const int32_t *>(d.P.p);
    const LinkMap *maps = reinterpret_cast<const LinkMap *>(d.link_map.p);
    const int32_t nl = (int32_t)d.n_links;
    int32_t *err = reinterpret_cast<int32_t *>(d.err.p);
    const bool bc = nl > 0;
    if (d.checked) {
        if (bc) aa_odd_kernel<Q, ST, 1, true, true><<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, 0, nullptr, nullptr);
        else aa_odd_kernel<Q, ST, 1, false, true><<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, 0, nullptr, nullptr);
        return cudaGetLastError();
    }
    // variant 4: slots from the 16-bit link codes, with the L2 prefetch of the codes
    if (sh.variant == 4) {
        const uint16_t *code = reinterpret_cast<const uint16_t *>(d.code.p);
        const int32_t *cb = reinterpret_cast<const int32_t *>(d.code_base.p);
        auto kc = sh.cells == 1
                      ? (bc ? aa_odd_kernel<Q, ST, 1, true, false, false, true> : aa_odd_kernel<Q, ST, 1, false, false, false, true>)
                      : (bc ? aa_odd_kernel<Q, ST, 2, true, false, false, true> : aa_odd_kernel<Q, ST, 2, false, false, false, true>);
        const int32_t pfc = (int32_t)persistent_grid(kc, sh.threads, INT32_MAX);
        kc<<<grid(sh.cells), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pfc, code, cb);
        return cudaGetLastError();
    }
    // hybrid cell order: the full bricks by arithmetic and their face lists,
    // the other cells (numbered after them) with the plain odd kernel
    if (d.order == SLBM_ORDER_HYBRID && d.n_full_cells > 0) {
        const int32_t nfull = (int32_t)d.n_full_cells;
        auto kf = bc ? aa_odd_brick_kernel<Q, ST, true> : aa_odd_brick_kernel<Q, ST, false>;
        const int32_t pff = (int32_t)persistent_grid(kf, 128, INT32_MAX);
        kf<<<(unsigned)((nfull + 127) / 128), 128, 0, st>>>(pdf, reinterpret_cast<const int32_t *>(d.face.p), S, nfull,
                                                             maps, p, pff);
        if (nf > nfull) {
            auto kr = bc ? aa_odd_kernel_from<Q, ST, true> : aa_odd_kernel_from<Q, ST, false>;
            const int32_t pfr = (int32_t)persistent_grid(kr, 128, INT32_MAX);
            kr<<<(unsigned)((nf - nfull + 127) / 128), 128, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pfr, nfull);
        }
        return cudaGetLastError();
    }
    // variant 6: every read of a tile staged in shared memory (index rows, own
    // rows, neighbour windows) by the bulk-copy engine, `cells` stages
    if (sh.variant == 6) {
        if (!d.win_tab.p) return cudaErrorInvalidValue;
        return bc ? launch_window<Q, ST, true>(d, sh.cells, st) : launch_window<Q, ST, false>(d, sh.cells, st);
    }
    // variant 5: variant 2 held to 64 registers a thread (more resident warps)
    if (sh.variant == 5) {
        auto kb = bc ? aa_odd_kernel_r64<Q, ST, true> : aa_odd_kernel_r64<Q, ST, false>;
        const int32_t pfb = (int32_t)persistent_grid(kb, sh.threads, INT32_MAX);
        kb<<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pfb);
        return cudaGetLastError();
    }
    // variant 3: slots re-read before the scatter (no links), with the L2 prefetch
    if (sh.variant == 3 && !bc) {
        auto kr = aa_odd_kernel<Q, ST, 1, false, false, true>;
        const int32_t pfr = (int32_t)persistent_grid(kr, sh.threads, INT32_MAX);
        kr<<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pfr, nullptr, nullptr);
        return cudaGetLastError();
    }
    // variant 2: L2 prefetch of the index rows one residency wave ahead
    int32_t pf = 0;
    if (sh.variant == 2 || sh.variant == 3) {
        auto kp = sh.cells == 1 ? (bc ? aa_odd_kernel<Q, ST, 1, true, false> : aa_odd_kernel<Q, ST, 1, false, false>)
                                : (bc ? aa_odd_kernel<Q, ST, 2, true, false> : aa_odd_kernel<Q, ST, 2, false, false>);
        pf = (int32_t)persistent_grid(kp, sh.threads, INT32_MAX);
    }
    switch (sh.cells * 2 + (bc ? 1 : 0)) {
        case 2: aa_odd_kernel<Q, ST, 1, false, false><<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pf, nullptr, nullptr); break;
        case 3: aa_odd_kernel<Q, ST, 1, true, false><<<grid(1), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pf, nullptr, nullptr); break;
        case 4: aa_odd_kernel<Q, ST, 2, false, false><<<grid(2), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pf, nullptr, nullptr); break;
        case 5: aa_odd_kernel<Q, ST, 2, true, false><<<grid(2), sh.threads, 0, st>>>(pdf, P, S, nf, maps, nl, p, err, pf, nullptr, nullptr); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace slbm
