// api.cu -- the extern "C" entry points declared in include/sparse_lbm.h.
//
// Host orchestration only: validation, memory, streams, CUDA graphs and
// copies.  Every arithmetic step of the method runs in the kernels of
// lists.cu, aa_*.cu, macro.cu and dense.cu.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace slbm {

static thread_local std::string g_msg;
static thread_local slbm_status g_status = SLBM_OK;

void set_error(slbm_status s, const std::string &msg) {
    g_status = s;
    g_msg = msg;
}
slbm_status last_status() { return g_status; }

int Ctx::alloc(DevBuf &b, int64_t bytes) {
    b.p = nullptr;
    b.bytes = 0;
    if (bytes <= 0) return 0;
    void *p = nullptr;
    if (hook) {
        p = hook->alloc((size_t)bytes, hook->ctx);
        if (!p) {
            fail(SLBM_ENOMEM, "allocator hook returned NULL");
            return -1;
        }
    } else {
        const cudaError_t e = cudaMalloc(&p, (size_t)bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(SLBM_ENOMEM, (std::string("cudaMalloc: ") + cudaGetErrorString(e)).c_str());
            return -1;
        }
    }
    b.p = p;
    b.bytes = bytes;
    if (held) *held += bytes;
    return 0;
}

void Ctx::release(DevBuf &b) {
    if (b.p) {
        if (hook) hook->free(b.p, hook->ctx);
        else cudaFree(b.p);
        if (held) *held -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

int Ctx::check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return 0;
    cudaGetLastError();
    fail(SLBM_ECUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return -1;
}

void Ctx::fail(slbm_status s, const char *msg) {
    if (status == SLBM_OK) {
        status = s;
        set_error(s, msg);
    }
}

CollideParams Domain::collide_params() const {
    CollideParams p{};
    p.omega_p = (float)omega_p;
    p.omega_m = (float)omega_m;
    p.fx = (float)force[0];
    p.fy = (float)force[1];
    p.fz = (float)force[2];
    const int s = storage == SLBM_FP32 ? 0 : scale_exp;
    p.scale = std::ldexp(1.0f, s);
    p.inv_scale = std::ldexp(1.0f, -s);
    const double sigma = std::ldexp(1.0, s), kp = 1.0 - 0.5 * omega_p, km = 1.0 - 0.5 * omega_m;
    p.kp = (float)kp;
    for (int m = 0; m < MAX_PAIRS; ++m) {
        p.alpha[m] = 0.f;
        p.kappa[m] = 0.f;
        if (2 * m + 1 >= q) continue;
        const int i = 2 * m + 1;
        const double w = q == 19 ? (double)wgt<19>(i) : (double)wgt<27>(i);
        const double cF = cx(i) * force[0] + cy(i) * force[1] + cz(i) * force[2];
        p.alpha[m] = (float)(sigma * kp * 9.0 * w * cF);
        p.kappa[m] = (float)(sigma * km * 3.0 * w * cF);
    }
    for (int a = 0; a < 19; ++a) p.mrt[a] = (float)mrt_rates[a];
    return p;
}

// Default launch shapes of a domain's operator, storage and links (called
// once its lists exist).  Even step: cells collided in pairs (measured faster
// except for FP16 MRT and untimed BF16); FP16 D3Q27 from bulk-staged tiles;
// the central-moment and cumulant collisions 64 x 1 (16-bit: 64 x 2).  Odd
// step: 128 x 1 with the L2 index prefetch (MRT: register-bounded;
// central-moment and cumulant: 256 x 1); D3Q19 and D3Q27 as below.  All measured fastest on the 256^3
// porosity-0.5 domain and, with links, on the particle bed.
static void default_shapes(Domain &d) {
    d.shape[0] = LaunchShape{64, 2, 0};
    d.shape[1] = LaunchShape{128, 1, 2};
    if (d.layout != SLBM_LAYOUT_SPARSE) return;
    if (d.op == SLBM_CM || d.op == SLBM_CUMULANT) {
        d.shape[0] = d.storage == SLBM_FP32 ? LaunchShape{64, 1, 0} : LaunchShape{64, 2, 0};
        d.shape[1] = LaunchShape{256, 1, 2};
    } else if (d.op == SLBM_MRT) {                                // paired even step in FP32
        if (d.storage == SLBM_FP32) d.shape[0] = LaunchShape{64, 2, 2};
        d.shape[1] = LaunchShape{128, 1, 5};
    } else if (d.storage != SLBM_BF16) {
        const bool f16 = d.storage == SLBM_FP16, links = d.n_links > 0;
        d.shape[0] = LaunchShape{64, 4, 2};
        if (d.q == 19) {
            // FP32 without links: two cells a thread (the link maps would hold
            // both cells' entries through the collision)
            d.shape[1] = f16 ? LaunchShape{256, 1, 2} : links ? LaunchShape{128, 1, 2} : LaunchShape{128, 2, 2};
        } else {
            // D3Q27: the FP16 even step with links from bulk-staged tiles (2
            // stages); odd step 256 x 1 (FP16: 256 x 2) without links, 64 x 1
            // (FP16: 128 x 1 register-bounded) with them
            if (f16 && links) d.shape[0] = LaunchShape{128, 2, 1};
            if (links) d.shape[1] = f16 ? LaunchShape{128, 1, 5} : LaunchShape{64, 1, 2};
            else d.shape[1] = f16 ? LaunchShape{256, 2, 2} : LaunchShape{256, 1, 2};
        }
    }
    if (d.order == SLBM_ORDER_HYBRID) d.shape[1] = LaunchShape{128, 1, 2};   // its one odd shape
}

// d'Humieres et al. (2002) rates with omega on the stress moments.
static void default_mrt_rates(Domain &d) {
    const double w = d.omega_p;
    const double r[19] = {0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, w, 1.4, w, 1.4, w, w, w, 1.98, 1.98, 1.98};
    for (int a = 0; a < 19; ++a) d.mrt_rates[a] = r[a];
}

template <int Q>
cudaError_t launch_aa_step_q(const Domain &d, int parity, cudaStream_t st);
extern template cudaError_t launch_aa_step_q<19>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_aa_step_q<27>(const Domain &, int, cudaStream_t);

cudaError_t launch_aa_step(const Domain &d, int parity, cudaStream_t st) {
    return d.q == 19 ? launch_aa_step_q<19>(d, parity, st) : launch_aa_step_q<27>(d, parity, st);
}

template <int Q>
cudaError_t launch_bc_fixup_q(const Domain &d, int post, cudaStream_t st);
extern template cudaError_t launch_bc_fixup_q<19>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_bc_fixup_q<27>(const Domain &, int, cudaStream_t);

cudaError_t launch_bc_fixup(const Domain &d, int post, cudaStream_t st) {
    return d.q == 19 ? launch_bc_fixup_q<19>(d, post, st) : launch_bc_fixup_q<27>(d, post, st);
}

// Step t -> t+1 (t = absolute step index).
static cudaError_t launch_one_step(const Domain &d, int64_t t, cudaStream_t st) {
    if (d.pull()) return launch_pull_step(d, t, st);
    return d.layout == SLBM_LAYOUT_SPARSE ? launch_aa_step(d, (int)(t & 1), st) : launch_dense_step(d, (int)(t & 1), st);
}

// The domain's cached graph of n steps from its current parity (pull layout:
// a separate one from step 0, whose first launch collides in place),
// captured on first use (capture records launches only; it runs nothing).
cudaError_t domain_graph(Domain &d, int32_t n, cudaGraphExec_t *out) {
    const std::pair<int, int> key(n, (d.pull() && d.step == 0) ? 2 : (int)(d.step & 1));
    auto it = d.graphs.find(key);
    if (it == d.graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(d.stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t le = cudaSuccess;
        for (int32_t t = 0; t < n && le == cudaSuccess; ++t) le = launch_one_step(d, d.step + t, d.stream);
        e = cudaStreamEndCapture(d.stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return le;
        }
        if (e != cudaSuccess) return e;
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        it = d.graphs.emplace(key, ex).first;
    }
    *out = it->second;
    return cudaSuccess;
}

static void drop_graphs(Domain &d) {
    for (auto &kv : d.graphs) cudaGraphExecDestroy(kv.second);
    d.graphs.clear();
}

static void release_all(Domain &d) {
    Ctx cx = d.ctx();
    DevBuf *bufs[] = {&d.pdf,  &d.pdf2,   &d.P,         &d.code,      &d.code_base, &d.win_tab, &d.win_code, &d.face, &d.cell_voxel, &d.link_cell,
                      &d.link_dir, &d.link_type, &d.link_map, &d.bcell, &d.bfirst, &d.bc_ubuf, &d.ltile,
                      &d.mask, &d.red_partial, &d.red_out, &d.err};
    for (DevBuf *b : bufs) cx.release(*b);
}

static slbm_status ok() {
    g_status = SLBM_OK;
    g_msg.clear();
    return SLBM_OK;
}

static slbm_status err(slbm_status s, const std::string &m) {
    set_error(s, m);
    return s;
}

// Build the 16-bit link codes on first use (sparse layout only).
static slbm_status ensure_codes(Domain &d) {
    if (d.layout != SLBM_LAYOUT_SPARSE) return err(SLBM_EUNSUPPORTED, "link codes exist for the sparse layout only");
    if (d.code.p || d.S == 0) return SLBM_OK;
    Ctx cx = d.ctx();
    if (build_link_codes(cx, d) || cx.check(cudaStreamSynchronize(d.stream), "build codes")) {
        cx.release(d.code);
        cx.release(d.code_base);
        return cx.status == SLBM_OK ? err(SLBM_ECUDA, g_msg) : cx.status;
    }
    return SLBM_OK;
}

// Build the neighbour-window table of the staged odd step on first use
// (sparse layout only).
static slbm_status ensure_window(Domain &d) {
    if (d.layout != SLBM_LAYOUT_SPARSE) return err(SLBM_EUNSUPPORTED, "the staged odd step exists for the sparse layout only");
    if (d.win_tab.p || d.S == 0) return SLBM_OK;
    Ctx cx = d.ctx();
    if (build_window_tab(cx, d) || cx.check(cudaStreamSynchronize(d.stream), "build window table")) {
        cx.release(d.win_tab);
        cx.release(d.win_code);
        return cx.status == SLBM_OK ? err(SLBM_ECUDA, g_msg) : cx.status;
    }
    return SLBM_OK;
}

static slbm_status cuda_err(cudaError_t e, const char *what) {
    cudaGetLastError();
    return err(SLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace slbm

using namespace slbm;

extern "C" {

const char *sparse_lbm_last_error(void) { return g_msg.c_str(); }

slbm_status sparse_lbm_create(const slbm_desc *desc, const slbm_allocator *alloc, void *stream, slbm_t **out) {
    const Range range_("slbm create");
    if (!desc || !out) return err(SLBM_EINVAL, "desc and out must be non-NULL");
    *out = nullptr;
    const slbm_desc &s = *desc;
    if (s.nx < 1 || s.ny < 1 || s.nz < 1) return err(SLBM_EINVAL, "nx, ny, nz must be >= 1");
    const int64_t N = (int64_t)s.nx * s.ny * s.nz;
    if (N >= ((int64_t)1 << 31)) return err(SLBM_EUNSUPPORTED, "nx*ny*nz must be < 2^31");
    if (!s.flags) return err(SLBM_EINVAL, "flags must be non-NULL");
    if (s.q != 19 && s.q != 27) return err(SLBM_EINVAL, "q must be 19 or 27");
    if (s.op < SLBM_SRT || s.op > SLBM_CUMULANT) return err(SLBM_EINVAL, "op must be SRT, TRT, MRT, CM or CUMULANT");
    if (s.op == SLBM_MRT && (s.q != 19 || s.layout == SLBM_LAYOUT_DENSE))
        return err(SLBM_EUNSUPPORTED, "MRT is built for D3Q19 sparse and pull layouts");
    if ((s.op == SLBM_CM || s.op == SLBM_CUMULANT) && (s.q != 27 || s.layout == SLBM_LAYOUT_DENSE))
        return err(SLBM_EUNSUPPORTED, "the central-moment and cumulant operators are built for D3Q27 sparse and pull "
                                      "layouts");
    if (!(s.omega_plus > 0.0 && s.omega_plus < 2.0)) return err(SLBM_EINVAL, "omega_plus must lie in (0, 2)");
    if (s.op == SLBM_TRT && !(s.trt_magic > 0.0 && std::isfinite(s.trt_magic)))
        return err(SLBM_EINVAL, "trt_magic must be > 0");
    if (s.storage < SLBM_FP32 || s.storage > SLBM_BF16) return err(SLBM_EINVAL, "storage must be 0, 1 or 2");
    if (s.scale_exp < -40 || s.scale_exp > 40) return err(SLBM_EINVAL, "scale_exp must lie in [-40, 40]");
    if (s.layout != SLBM_LAYOUT_SPARSE && s.layout != SLBM_LAYOUT_DENSE && s.layout != SLBM_LAYOUT_SPARSE_PULL)
        return err(SLBM_EINVAL, "bad layout");
    if (s.order != SLBM_ORDER_LEX && s.order != SLBM_ORDER_BRICK8 && s.order != SLBM_ORDER_HYBRID)
        return err(SLBM_EINVAL, "order must be 0, 1 or 2");
    if (s.order != SLBM_ORDER_LEX && s.layout == SLBM_LAYOUT_DENSE)
        return err(SLBM_EUNSUPPORTED, "the dense layout has no cell order");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(s.force[a])) return err(SLBM_EINVAL, "force must be finite");
    if (!(s.rho_out > 0.0 && std::isfinite(s.rho_out))) return err(SLBM_EINVAL, "rho_out must be > 0");
    // host pass over the flags: range check, boundary presence, counts
    int64_t n_fluid_host = 0, n_inlet = 0;
    bool has_bc = false;
    for (int64_t v = 0; v < N; ++v) {
        const uint8_t f = s.flags[v];
        if (f > 3) return err(SLBM_EINVAL, "flag values must be 0..3");
        n_fluid_host += f == 0;
        n_inlet += f == 2;
        has_bc |= f >= 2;
    }
    if (s.inlet_u && s.n_inlet_u != n_inlet)
        return err(SLBM_EINVAL, "n_inlet_u must equal the number of inlet voxels");
    if (s.layout == SLBM_LAYOUT_DENSE && has_bc)
        return err(SLBM_EUNSUPPORTED, "the dense comparator supports walls and periodic boundaries only");
    if (s.layout == SLBM_LAYOUT_SPARSE_PULL && has_bc)
        return err(SLBM_EUNSUPPORTED, "the pull layout supports walls and periodic boundaries only");
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return err(SLBM_ECUDA, "no CUDA device available (there is no CPU fallback)");
    }

    slbm_t *h = new slbm_t();
    Domain &d = h->d;
    d.nx = s.nx;
    d.ny = s.ny;
    d.nz = s.nz;
    d.periodic = s.periodic & 7u;
    d.n_vox = N;
    d.q = s.q;
    d.op = s.op;
    d.storage = s.storage;
    d.layout = s.layout;
    d.order = s.order;
    d.scale_exp = s.storage == SLBM_FP32 ? 0 : s.scale_exp;
    d.omega_p = s.omega_plus;
    d.magic = s.trt_magic;
    d.omega_m = s.op == SLBM_TRT ? 1.0 / (s.trt_magic / (1.0 / s.omega_plus - 0.5) + 0.5) : s.omega_plus;
    if (d.op == SLBM_MRT) default_mrt_rates(d);
    if (d.op == SLBM_CM || d.op == SLBM_CUMULANT) {   // bulk and higher-order rates
        d.mrt_rates[0] = 1.0;
        d.mrt_rates[1] = 1.0;
    }
    for (int a = 0; a < 3; ++a) d.force[a] = s.force[a];
    d.rho_out = s.rho_out;
    if (alloc) {
        if (!alloc->alloc || !alloc->free) {
            delete h;
            return err(SLBM_EINVAL, "allocator needs alloc and free");
        }
        d.hook = *alloc;
        d.has_hook = true;
    }
    if (stream) {
        d.stream = (cudaStream_t)stream;
    } else {
        ce = cudaStreamCreate(&d.stream);
        if (ce != cudaSuccess) {
            delete h;
            return cuda_err(ce, "cudaStreamCreate");
        }
        d.own_stream = true;
    }
    Ctx cx = d.ctx();
    DevBuf flags;
    int rc = cx.alloc(flags, N);
    if (!rc) rc = cx.check(cudaMemcpyAsync(flags.p, s.flags, N, cudaMemcpyHostToDevice, d.stream), "flags H2D");
    if (!rc) {
        if (d.sparse()) {
            rc = build_sparse_lists(cx, d, (const uint8_t *)flags.p, has_bc, s.inlet_u, s.n_inlet_u);
            if (!rc && d.n_fluid != n_fluid_host) {
                cx.fail(SLBM_ECUDA, "device compaction count disagrees with the host count");
                rc = -1;
            }
            if (!rc && d.pull() && d.S > 0) {   // the pull step reads the canonical entries P(i,k)
                DevBuf canon;
                rc = cx.alloc(canon, (int64_t)(d.q - 1) * d.S * 4);
                if (!rc) rc = cx.check(launch_unflip(d, (int32_t *)canon.p, d.stream), "unflip");
                if (!rc) rc = cx.check(cudaStreamSynchronize(d.stream), "unflip sync");
                if (!rc) {
                    cx.release(d.P);
                    d.P = canon;
                } else {
                    cx.release(canon);
                }
            }
        } else {
            d.n_fluid = n_fluid_host;
            d.S = (N + 127) / 128 * 128;
            rc = build_dense_mask(cx, d, (const uint8_t *)flags.p);
        }
    }
    const int64_t rows_bytes = (int64_t)d.q * d.S * d.bytes_per_pdf();
    if (!rc) rc = cx.alloc(d.pdf, rows_bytes);
    if (!rc && rows_bytes) rc = cx.check(cudaMemsetAsync(d.pdf.p, 0, rows_bytes, d.stream), "memset pdf");
    if (!rc && d.pull()) rc = cx.alloc(d.pdf2, rows_bytes);
    if (!rc && d.pull() && rows_bytes) rc = cx.check(cudaMemsetAsync(d.pdf2.p, 0, rows_bytes, d.stream), "memset pdf2");
    if (!rc) rc = cx.alloc(d.red_partial, std::max<int64_t>(d.red_chunks(), 1) * (5 * sizeof(double) + 2 * sizeof(float)));
    if (!rc) rc = cx.alloc(d.red_out, 8 * sizeof(double));
    if (!rc) rc = cx.alloc(d.err, sizeof(int32_t));
    if (!rc) rc = cx.check(cudaMemsetAsync(d.err.p, 0, sizeof(int32_t), d.stream), "memset err");
    if (!rc) rc = cx.check(cudaStreamSynchronize(d.stream), "create sync");
    cx.release(flags);
    default_shapes(d);
    if (rc) {
        const slbm_status st = cx.status == SLBM_OK ? SLBM_ECUDA : cx.status;
        const std::string m = g_msg;
        release_all(d);
        if (d.own_stream) cudaStreamDestroy(d.stream);
        delete h;
        return err(st, m);
    }
    *out = h;
    return ok();
}

slbm_status sparse_lbm_step(slbm_t *h, int32_t n) {
    const Range range_("slbm step");
    if (!h || n < 0) return err(SLBM_EINVAL, "need a handle and n >= 0");
    Domain &d = h->d;
    for (int32_t t = 0; t < n; ++t) {
        const cudaError_t e = launch_one_step(d, d.step, d.stream);
        if (e != cudaSuccess) return cuda_err(e, "step launch");
        ++d.step;
    }
    return ok();
}

slbm_status sparse_lbm_step_graph(slbm_t *h, int32_t n) {
    const Range range_("slbm step (graph)");
    if (!h || n < 0) return err(SLBM_EINVAL, "need a handle and n >= 0");
    if (n == 0) return ok();
    Domain &d = h->d;
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = domain_graph(d, n, &ex);
    if (e != cudaSuccess) return cuda_err(e, "graph capture");
    e = cudaGraphLaunch(ex, d.stream);
    if (e != cudaSuccess) return cuda_err(e, "graph launch");
    d.step += n;
    return ok();
}

slbm_status sparse_lbm_macroscopic(slbm_t *h, float *rho, float *u, int32_t order, int32_t mem) {
    const Range range_("slbm macroscopic");
    if (!h) return err(SLBM_EINVAL, "null handle");
    if (order != SLBM_ORDER_CELLS && order != SLBM_ORDER_VOXELS) return err(SLBM_EINVAL, "bad order");
    if (mem != SLBM_MEM_DEVICE && mem != SLBM_MEM_HOST) return err(SLBM_EINVAL, "bad mem");
    Domain &d = h->d;
    const int64_t n = order == SLBM_ORDER_VOXELS ? d.n_vox : (d.sparse() ? d.n_fluid : d.n_vox);
    if (mem == SLBM_MEM_DEVICE) {
        if (order == SLBM_ORDER_VOXELS) {   // zero the non-fluid entries first
            if (rho && n) cudaMemsetAsync(rho, 0, n * sizeof(float), d.stream);
            if (u && n) cudaMemsetAsync(u, 0, 3 * n * sizeof(float), d.stream);
        }
        const cudaError_t e = launch_macroscopic(d, rho, u, order, d.stream);
        return e == cudaSuccess ? ok() : cuda_err(e, "macroscopic");
    }
    Ctx cx = d.ctx();
    cx.held = nullptr;
    DevBuf dr, du;
    if ((rho && cx.alloc(dr, n * sizeof(float))) || (u && cx.alloc(du, 3 * n * sizeof(float))))
        return err(cx.status, g_msg);
    int rc = 0;
    if (dr.p) rc |= cx.check(cudaMemsetAsync(dr.p, 0, n * sizeof(float), d.stream), "memset");
    if (du.p) rc |= cx.check(cudaMemsetAsync(du.p, 0, 3 * n * sizeof(float), d.stream), "memset");
    if (!rc) rc = cx.check(launch_macroscopic(d, (float *)dr.p, (float *)du.p, order, d.stream), "macroscopic");
    if (!rc && dr.p)
        rc = cx.check(cudaMemcpyAsync(rho, dr.p, n * sizeof(float), cudaMemcpyDeviceToHost, d.stream), "rho D2H");
    if (!rc && du.p)
        rc = cx.check(cudaMemcpyAsync(u, du.p, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, d.stream), "u D2H");
    if (!rc) rc = cx.check(cudaStreamSynchronize(d.stream), "macroscopic sync");
    cx.release(dr);
    cx.release(du);
    return rc ? err(cx.status, g_msg) : ok();
}

slbm_status sparse_lbm_reduce(slbm_t *h, double *out, int32_t mem) {
    const Range range_("slbm reduce");
    if (!h || !out) return err(SLBM_EINVAL, "null argument");
    Domain &d = h->d;
    if (mem == SLBM_MEM_DEVICE) {
        const cudaError_t e = launch_reduce(d, out, d.stream);
        return e == cudaSuccess ? ok() : cuda_err(e, "reduce");
    }
    if (mem != SLBM_MEM_HOST) return err(SLBM_EINVAL, "bad mem");
    cudaError_t e = launch_reduce(d, (double *)d.red_out.p, d.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d.red_out.p, 5 * sizeof(double), cudaMemcpyDeviceToHost, d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
    if (e != cudaSuccess) return cuda_err(e, "reduce");
    for (int c = 0; c < 5; ++c)
        if (!std::isfinite(out[c])) return err(SLBM_EDIVERGED, "domain sums are not finite");
    return ok();
}

slbm_status sparse_lbm_reduce_ext(slbm_t *h, double *out, int32_t mem) {
    const Range range_("slbm reduce ext");
    if (!h || !out) return err(SLBM_EINVAL, "null argument");
    Domain &d = h->d;
    if (mem == SLBM_MEM_DEVICE) {
        const cudaError_t e = launch_reduce_ext(d, out, d.stream);
        return e == cudaSuccess ? ok() : cuda_err(e, "reduce_ext");
    }
    if (mem != SLBM_MEM_HOST) return err(SLBM_EINVAL, "bad mem");
    cudaError_t e = launch_reduce_ext(d, (double *)d.red_out.p, d.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d.red_out.p, 7 * sizeof(double), cudaMemcpyDeviceToHost, d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
    if (e != cudaSuccess) return cuda_err(e, "reduce_ext");
    for (int c = 0; c < 7; ++c)
        if (!std::isfinite(out[c])) return err(SLBM_EDIVERGED, "domain sums or maxima are not finite");
    if (out[6] > 0.3) return err(SLBM_EDIVERGED, "a cell's speed exceeds 0.3");
    return ok();
}

slbm_status sparse_lbm_set_storage(slbm_t *h, int32_t storage, int32_t scale_exp) {
    const Range range_("slbm set storage");
    if (!h) return err(SLBM_EINVAL, "null handle");
    if (storage < SLBM_FP32 || storage > SLBM_BF16) return err(SLBM_EINVAL, "storage must be 0, 1 or 2");
    if (scale_exp < -40 || scale_exp > 40) return err(SLBM_EINVAL, "scale_exp must lie in [-40, 40]");
    Domain &d = h->d;
    if (!d.pools.empty()) return err(SLBM_EINVAL, "the domain is a pool member: remove it from its pool first");
    const int new_s = storage == SLBM_FP32 ? 0 : scale_exp;
    if (storage == d.storage && new_s == d.scale_exp) return ok();
    Ctx cx = d.ctx();
    if (convert_storage(cx, d, storage, new_s)) return err(cx.status == SLBM_OK ? SLBM_ECUDA : cx.status, g_msg);
    default_shapes(d);
    drop_graphs(d);
    return ok();
}

slbm_status sparse_lbm_init_equilibrium(slbm_t *h, const float *rho, const float *u, int32_t order, int32_t mem) {
    if (!h) return err(SLBM_EINVAL, "null handle");
    if (order != SLBM_ORDER_CELLS && order != SLBM_ORDER_VOXELS) return err(SLBM_EINVAL, "bad order");
    Domain &d = h->d;
    const int64_t n = order == SLBM_ORDER_VOXELS ? d.n_vox : (d.sparse() ? d.n_fluid : d.n_vox);
    Ctx cx = d.ctx();
    cx.held = nullptr;
    DevBuf dr, du;
    const float *pr = rho, *pu = u;
    int rc = 0;
    if (mem == SLBM_MEM_HOST) {
        if (rho && !rc) {
            rc = cx.alloc(dr, n * sizeof(float));
            if (!rc) rc = cx.check(cudaMemcpyAsync(dr.p, rho, n * sizeof(float), cudaMemcpyHostToDevice, d.stream), "H2D");
            pr = (const float *)dr.p;
        }
        if (u && !rc) {
            rc = cx.alloc(du, 3 * n * sizeof(float));
            if (!rc) rc = cx.check(cudaMemcpyAsync(du.p, u, 3 * n * sizeof(float), cudaMemcpyHostToDevice, d.stream), "H2D");
            pu = (const float *)du.p;
        }
    } else if (mem != SLBM_MEM_DEVICE) {
        return err(SLBM_EINVAL, "bad mem");
    }
    if (!rc) rc = cx.check(launch_init_equilibrium(d, pr, pu, order, d.stream), "init");
    if (!rc && mem == SLBM_MEM_HOST) rc = cx.check(cudaStreamSynchronize(d.stream), "init sync");
    cx.release(dr);
    cx.release(du);
    if (rc) return err(cx.status, g_msg);
    d.step = 0;
    return ok();
}

slbm_status sparse_lbm_info(const slbm_t *h, slbm_info *o) {
    if (!h || !o) return err(SLBM_EINVAL, "null argument");
    const Domain &d = h->d;
    o->n_voxels = d.n_vox;
    o->n_fluid = d.n_fluid;
    o->stride = d.S;
    o->n_bc_links = d.n_links;
    o->device_bytes = d.device_bytes;
    o->step = d.step;
    o->q = d.q;
    o->op = d.op;
    o->storage = d.storage;
    o->layout = d.layout;
    o->scale_exp = d.scale_exp;
    o->pad = 0;
    return ok();
}

slbm_status sparse_lbm_export_lists(const slbm_t *h, int32_t *cell_voxel, int32_t *index_rows, int32_t *link_cell,
                                    int32_t *link_dir, int32_t *link_type) {
    if (!h) return err(SLBM_EINVAL, "null handle");
    const Domain &d = h->d;
    if (!d.sparse()) return err(SLBM_EUNSUPPORTED, "lists exist for the sparse layouts only");
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, int64_t bytes) {
        if (dst && bytes > 0 && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, d.stream);
    };
    cp(cell_voxel, d.cell_voxel.p, d.n_fluid * 4);
    const int64_t pbytes = (int64_t)(d.q - 1) * d.S * 4;
    Ctx cx = const_cast<Domain &>(d).ctx();
    cx.held = nullptr;
    DevBuf tmp;
    if (index_rows && pbytes > 0) {
        if (d.pull()) {                 // stored canonical
            cp(index_rows, d.P.p, pbytes);
        } else {
            if (cx.alloc(tmp, pbytes)) return err(cx.status, g_msg);
            e = launch_unflip(d, (int32_t *)tmp.p, d.stream);
            cp(index_rows, tmp.p, pbytes);
        }
    }
    cp(link_cell, d.link_cell.p, d.n_links * 4);
    cp(link_dir, d.link_dir.p, d.n_links * 4);
    cp(link_type, d.link_type.p, d.n_links * 4);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
    cx.release(tmp);
    return e == cudaSuccess ? ok() : cuda_err(e, "export lists");
}

slbm_status sparse_lbm_export_codes(slbm_t *h, uint16_t *codes, int32_t *bases) {
    if (!h) return err(SLBM_EINVAL, "null handle");
    const slbm_status st = ensure_codes(h->d);
    if (st != SLBM_OK) return st;
    const Domain &d = h->d;
    cudaError_t e = cudaSuccess;
    const int64_t cbytes = (int64_t)(d.q - 1) * d.S * 2, bbytes = d.S / CODE_TILE * (d.q - 1) * 4;
    if (codes && cbytes > 0) e = cudaMemcpyAsync(codes, d.code.p, cbytes, cudaMemcpyDeviceToHost, d.stream);
    if (bases && bbytes > 0 && e == cudaSuccess)
        e = cudaMemcpyAsync(bases, d.code_base.p, bbytes, cudaMemcpyDeviceToHost, d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
    return e == cudaSuccess ? ok() : cuda_err(e, "export codes");
}

slbm_status sparse_lbm_state_bytes(const slbm_t *h, int64_t *bytes) {
    if (!h || !bytes) return err(SLBM_EINVAL, "null argument");
    *bytes = (int64_t)h->d.q * h->d.S * h->d.bytes_per_pdf();
    return ok();
}

slbm_status sparse_lbm_get_state(const slbm_t *h, void *host, int64_t *step) {
    if (!h || !host) return err(SLBM_EINVAL, "null argument");
    const Domain &d = h->d;
    const int64_t b = (int64_t)d.q * d.S * d.bytes_per_pdf();
    cudaError_t e = cudaSuccess;
    if (b) e = cudaMemcpyAsync(host, d.cur_pdf(), b, cudaMemcpyDeviceToHost, d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
    if (e != cudaSuccess) return cuda_err(e, "get_state");
    if (step) *step = d.step;
    return ok();
}

slbm_status sparse_lbm_set_state(slbm_t *h, const void *host, int64_t step) {
    if (!h || !host || step < 0) return err(SLBM_EINVAL, "bad argument");
    Domain &d = h->d;
    const int64_t b = (int64_t)d.q * d.S * d.bytes_per_pdf();
    cudaError_t e = cudaSuccess;
    const int64_t was = d.step;
    d.step = step;
    void *dst = d.cur_pdf();           // the grid that holds the state at `step`
    d.step = was;
    if (b) e = cudaMemcpyAsync(dst, host, b, cudaMemcpyHostToDevice, d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
    if (e != cudaSuccess) return cuda_err(e, "set_state");
    d.step = step;
    return ok();
}

slbm_status sparse_lbm_set_mrt_rates(slbm_t *h, const double *rates) {
    if (!h || !rates) return err(SLBM_EINVAL, "null argument");
    Domain &d = h->d;
    if (d.op != SLBM_MRT) return err(SLBM_EINVAL, "not an MRT domain");
    for (int a = 0; a < 19; ++a) {
        if (a == 0 || a == 3 || a == 5 || a == 7) continue;
        if (!(rates[a] > 0.0 && rates[a] < 2.0)) return err(SLBM_EINVAL, "MRT rates must lie in (0, 2)");
    }
    for (int a = 0; a < 19; ++a) d.mrt_rates[a] = (a == 0 || a == 3 || a == 5 || a == 7) ? 0.0 : rates[a];
    drop_graphs(d);
    return ok();
}

slbm_status sparse_lbm_set_cm_rates(slbm_t *h, double bulk, double higher) {
    if (!h) return err(SLBM_EINVAL, "null handle");
    Domain &d = h->d;
    if (d.op != SLBM_CM && d.op != SLBM_CUMULANT) return err(SLBM_EINVAL, "not a central-moment or cumulant domain");
    if (!(bulk > 0.0 && bulk <= 2.0) || !(higher > 0.0 && higher <= 2.0))
        return err(SLBM_EINVAL, "rates must lie in (0, 2]");
    if (d.op == SLBM_CUMULANT && higher != 1.0)
        return err(SLBM_EUNSUPPORTED, "the cumulant collision is built with the higher-order rate 1");
    d.mrt_rates[0] = bulk;
    d.mrt_rates[1] = higher;
    drop_graphs(d);
    return ok();
}

slbm_status sparse_lbm_set_launch(slbm_t *h, int32_t parity, int32_t threads, int32_t cells, int32_t variant) {
    if (!h || (parity != 0 && parity != 1)) return err(SLBM_EINVAL, "bad handle or parity");
    if (h->d.pull()) return err(SLBM_EUNSUPPORTED, "the pull layout has one launch shape");
    const bool moment = h->d.op == SLBM_MRT || h->d.op == SLBM_CM || h->d.op == SLBM_CUMULANT;
    if (moment) {
        // even: 0, 2 (MRT pairs), 5; odd: 0, 2, 3 (no links), 5 -- 5 is 128 x 1 only
        const bool okv = parity == 0 ? (variant == 0 || variant == 5 || (h->d.op == SLBM_MRT && variant == 2))
                                     : (variant == 0 || variant == 2 || variant == 3 || variant == 5);
        if (!okv)
            return err(SLBM_EUNSUPPORTED, "MRT, central-moment and cumulant domains run even variants 0 and 5 "
                                          "(MRT also 2) and odd variants 0, 2, 3 and 5");
        if (parity == 0 && cells == 4)
            return err(SLBM_EUNSUPPORTED, "MRT, central-moment and cumulant even step: 1 or 2 cells per thread");
        if (parity == 1 && variant == 3 && h->d.n_links > 0)
            return err(SLBM_EUNSUPPORTED, "odd variant 3 (slots re-read) covers domains without inlet/outlet links");
        if (variant == 5) {
            if (threads != 128 || cells != 1)
                return err(SLBM_EINVAL, "variant 5 of the moment-space operators: 128 threads, 1 cell each");
            h->d.shape[parity] = LaunchShape{threads, cells, variant};
            drop_graphs(h->d);
            return ok();
        }
    }
    if (parity == 1 && h->d.order == SLBM_ORDER_HYBRID && h->d.layout == SLBM_LAYOUT_SPARSE &&
        !(threads == 128 && cells == 1 && variant == 2))
        return err(SLBM_EUNSUPPORTED, "the hybrid cell order has one odd-step shape (full bricks + 128 x 1, variant 2)");
    if (variant == 0) {
        if (threads < 32 || threads > 256 || threads % 32)
            return err(SLBM_EINVAL, "threads must be 32..256, multiple of 32");
        const bool okc = parity == 0 ? (cells == 1 || cells == 2 || cells == 4) : (cells == 1 || cells == 2);
        if (!okc) return err(SLBM_EINVAL, "cells per thread: even 1/2/4, odd 1/2");
    } else if (variant == 1) {
        if (h->d.layout != SLBM_LAYOUT_SPARSE || h->d.storage == SLBM_BF16)
            return err(SLBM_EUNSUPPORTED, "the staged variant covers sparse FP32/FP16 domains");
        if ((threads != 64 && threads != 128) || (cells != 2 && cells != 4))
            return err(SLBM_EINVAL, "staged variant: tile 64 or 128, stages 2 or 4");
    } else if (parity == 0 && variant == 2) {
        if (threads < 32 || threads > 256 || threads % 32 || (cells != 2 && cells != 4))
            return err(SLBM_EINVAL, "even variant 2 (paired collision): threads 32..256 (multiple of 32), "
                                    "cells 2 or 4");
    } else if (parity == 0 && variant == 3) {
        if (h->d.layout != SLBM_LAYOUT_SPARSE || h->d.storage == SLBM_BF16)
            return err(SLBM_EUNSUPPORTED, "the staged variants cover sparse FP32/FP16 domains");
        if ((threads != 64 && threads != 128) || (cells != 2 && cells != 4))
            return err(SLBM_EINVAL, "staged variant: tile 64 or 128, stages 2 or 4");
    } else if (parity == 1 && variant == 6) {
        if (h->d.layout != SLBM_LAYOUT_SPARSE) return err(SLBM_EUNSUPPORTED, "the staged odd step covers sparse domains");
        if (threads != 128 || cells < 2 || cells > 4)
            return err(SLBM_EINVAL, "odd variant 6: 128 threads (one tile of cells), 2..4 stages");
        const slbm_status st = ensure_window(h->d);
        if (st != SLBM_OK) return st;
    } else if (parity == 1 && variant >= 2 && variant <= 5) {
        if (threads < 32 || threads > 256 || threads % 32 || (cells != 1 && !((variant == 2 || variant == 4) && cells == 2)))
            return err(SLBM_EINVAL, "odd variants 2..5: threads 32..256 (multiple of 32), "
                                    "cells 1 (variants 2 and 4 also 2)");
        if (variant == 4) {
            const slbm_status st = ensure_codes(h->d);
            if (st != SLBM_OK) return st;
        }
    } else {
        return err(SLBM_EINVAL, "variant must be 0..3 (even step) or 0..6 (odd step)");
    }
    h->d.shape[parity] = LaunchShape{threads, cells, variant};
    drop_graphs(h->d);
    return ok();
}

slbm_status sparse_lbm_set_checked(slbm_t *h, int32_t on) {
    if (!h) return err(SLBM_EINVAL, "null handle");
    h->d.checked = on != 0;
    drop_graphs(h->d);
    return ok();
}

slbm_status sparse_lbm_device_error(slbm_t *h, int32_t *code) {
    if (!h || !code) return err(SLBM_EINVAL, "null argument");
    Domain &d = h->d;
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, d.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, d.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err.p, 0, sizeof(int32_t), d.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d.stream);
    if (e != cudaSuccess) return cuda_err(e, "device_error");
    *code = v;
    return v ? err(SLBM_EDEVICE, "a checked kernel latched an out-of-range slot") : ok();
}

void sparse_lbm_free(slbm_t *h) {
    if (!h) return;
    Domain &d = h->d;
    for (::slbm_pool *p : d.pools) pool_forget_member(p, h);   // no pool keeps a dangling member
    d.pools.clear();
    cudaStreamSynchronize(d.stream);
    drop_graphs(d);
    release_all(d);
    if (d.own_stream) cudaStreamDestroy(d.stream);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
