// internal.h -- host-side structures shared by the library's translation units.
#pragma once

#include <algorithm>
#include <map>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "sparse_lbm.h"

namespace slbm {

// Named NVTX range for profilers (Nsight); free when no tool is attached.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Thread-local error record behind sparse_lbm_last_error().
void set_error(slbm_status s, const std::string &msg);
slbm_status last_status();

struct DevBuf {
    void *p = nullptr;
    int64_t bytes = 0;
};

// Allocation / error context of one API call on one domain.
struct Ctx {
    cudaStream_t stream = nullptr;
    const slbm_allocator *hook = nullptr;
    int64_t *held = nullptr;        // running total of bytes owned by the domain
    slbm_status status = SLBM_OK;

    int alloc(DevBuf &b, int64_t bytes);
    void release(DevBuf &b);
    int check(cudaError_t e, const char *what);
    void fail(slbm_status s, const char *msg);
};

// variant 0: one thread per `cells` consecutive cells, `threads` per block.
// variant 1: persistent CTAs of `threads` (= tile) cells with `cells` (=
// pipeline stages) bulk-staged tiles in flight.
struct LaunchShape {
    int32_t threads;
    int32_t cells;
    int32_t variant;
};

struct Domain {
    // problem
    int32_t nx = 0, ny = 0, nz = 0;
    uint32_t periodic = 0;
    int64_t n_vox = 0;
    int32_t q = 19, op = SLBM_SRT, storage = SLBM_FP32, layout = SLBM_LAYOUT_SPARSE, scale_exp = 0;
    int32_t order = SLBM_ORDER_LEX;    // compacted cell order
    double omega_p = 1.0, omega_m = 1.0, magic = 0.1875, force[3] = {0, 0, 0}, rho_out = 1.0;
    double mrt_rates[19] = {};         // MRT: rate of each basis moment
    // sizes
    int64_t n_fluid = 0, S = 0, n_links = 0, step = 0;
    // device data
    DevBuf pdf;                        // Q x S stored populations
    DevBuf pdf2;                       // second grid (pull layout only)
    DevBuf P;                          // (Q-1) x S odd-step slots R(i,k) (row-flipped pull entries)
    DevBuf code;                       // (Q-1) x S 16-bit link codes of R (sparse)
    DevBuf code_base;                  // (S / CODE_TILE) x (Q-1) column bases of the codes
    DevBuf win_tab;                    // (S / 128) x (Q-1) neighbour windows of the staged odd step
    DevBuf win_code;                   // (Q-1) x S 16-bit staged positions of R (staged odd step)
    DevBuf face;                       // face links of the full bricks (hybrid order)
    int64_t n_full_cells = 0;          // hybrid order: cells of the full bricks (512 each), numbered first
    DevBuf cell_voxel;                 // N_F voxel ids (sparse)
    DevBuf link_cell, link_dir, link_type, link_map;   // boundary links (sparse)
    DevBuf bcell, bfirst, bc_ubuf;     // cells with links: id, first link (n+1), saved velocity
    DevBuf ltile;                      // first link of each 32-cell tile (n_tiles + 1)
    int64_t n_bcells = 0;
    DevBuf mask;                       // per-voxel link mask (dense)
    DevBuf red_partial;                // per-chunk FP64 partial sums (5 doubles), then per-chunk maxima (2 floats)
    DevBuf red_out;                    // 8 doubles
    DevBuf err;                        // latched device error word
    // execution
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    slbm_allocator hook{};
    bool has_hook = false;
    int64_t device_bytes = 0;
    LaunchShape shape[2] = {{64, 2, 0}, {128, 1, 2}};
    bool checked = false;
    std::vector<::slbm_pool *> pools;  // pools that hold this domain as a member
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (n, parity) -> exec

    int bytes_per_pdf() const { return storage == SLBM_FP32 ? 4 : 2; }
    bool sparse() const { return layout != SLBM_LAYOUT_DENSE; }      // compacted cell lists
    bool pull() const { return layout == SLBM_LAYOUT_SPARSE_PULL; }
    // grid holding the current state (pull: A at t = 0 and odd t, else B)
    void *cur_pdf() const { return (pull() && step > 0 && !(step & 1)) ? pdf2.p : pdf.p; }
    int64_t red_chunks() const;
    CollideParams collide_params() const;
    Ctx ctx() {
        Ctx c;
        c.stream = stream;
        c.hook = has_hook ? &hook : nullptr;
        c.held = &device_bytes;
        return c;
    }
};

// Chunking of the deterministic reductions: fixed cells per chunk.
constexpr int RED_THREADS = 256;
constexpr int RED_CELLS_PER_THREAD = 8;
constexpr int RED_CHUNK = RED_THREADS * RED_CELLS_PER_THREAD;

// lists.cu
cudaError_t launch_unflip(const Domain &d, int32_t *out, cudaStream_t st);
// 16-bit link codes of the odd-step slots (after build_sparse_lists)
int build_link_codes(Ctx &cx, Domain &d);
// neighbour-window table of the staged odd step (launch variant 6)
int build_window_tab(Ctx &cx, Domain &d);
int build_sparse_lists(Ctx &cx, Domain &d, const uint8_t *d_flags, bool has_bc, const float *h_inlet_u,
                       int64_t n_inlet_u);
// aa_q19.cu / aa_q27.cu (dispatch in api.cu)
cudaError_t launch_aa_step(const Domain &d, int parity, cudaStream_t st);
// pull.cu: one two-grid pull step from step index d.step + t
cudaError_t launch_pull_step(const Domain &d, int64_t t, cudaStream_t st);
// boundary fix-up before (post = 0) / after (post = 1) an even step
cudaError_t launch_bc_fixup(const Domain &d, int post, cudaStream_t st);
// The domain's cached CUDA graph of n steps from its current parity (captured
// on first use); launch it on any stream.
cudaError_t domain_graph(Domain &d, int32_t n, cudaGraphExec_t *out);
// macro.cu
cudaError_t launch_macroscopic(const Domain &d, float *rho, float *u, int order, cudaStream_t st);
cudaError_t launch_reduce(const Domain &d, double *out_dev, cudaStream_t st);
// the five sums plus max |f_i - w_i| and max |u| (7 doubles)
cudaError_t launch_reduce_ext(const Domain &d, double *out_dev, cudaStream_t st);
cudaError_t launch_init_equilibrium(const Domain &d, const float *rho, const float *u, int order,
                                    cudaStream_t st);
// convert.cu: stored populations to another storage format / scale
int convert_storage(Ctx &cx, Domain &d, int storage, int scale_exp);
// pool.cu: take a domain that is being freed out of a pool's member slots
void pool_forget_member(::slbm_pool *p, ::slbm_domain *h);
// dense.cu
int build_dense_mask(Ctx &cx, Domain &d, const uint8_t *d_flags);
cudaError_t launch_dense_step(const Domain &d, int parity, cudaStream_t st);

}  // namespace slbm

struct slbm_domain {
    slbm::Domain d;
};
