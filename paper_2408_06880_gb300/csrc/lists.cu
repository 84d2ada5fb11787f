// lists.cu -- device construction of the sparse data structure (Sec. 3.1):
// compaction of fluid voxels into the PDF-list order, the pull index-list with
// no-slip / periodic folded in (Sec. 3.1.1), and the inlet/outlet link table.
//
// The compaction is an exclusive prefix sum of (flag == fluid) over voxel ids,
// so cell k is the k-th fluid voxel in ascending id: exactly the order of a
// sequential scan, whatever the launch shape (integer sums are exact).
#include "aa_window.cuh"
#include "brick.cuh"
#include "internal.h"

namespace slbm {

// ------------------------------------------------------------ block scan
// Three-phase exclusive scan of an int-valued sequence produced by a functor:
//   1. per-tile totals, 2. exclusive scan of the totals (one block),
//   3. per-tile rescan that emits every element's exclusive prefix.
// A tile is SCAN_THREADS x SCAN_ITEMS consecutive elements; thread t owns
// elements [t*ITEMS, (t+1)*ITEMS) of its tile.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int32_t block_exclusive_sum(int32_t v, int32_t *smem_warp, int32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int32_t s = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) smem_warp[lane] = s;   // inclusive warp prefix
    }
    __syncthreads();
    total = smem_warp[(blockDim.x >> 5) - 1];
    const int32_t warp_base = warp > 0 ? smem_warp[warp - 1] : 0;
    __syncthreads();
    return warp_base + x - v;
}

template <class Fn>
__global__ void scan_tile_totals(Fn fn, int64_t n, int32_t *tile_total) {
    __shared__ int32_t sw[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < n) s += fn.value(base + j);
    int32_t tot;
    block_exclusive_sum(s, sw, tot);
    if (threadIdx.x == 0) tile_total[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile totals in place; grand total out.
__global__ void scan_tile_offsets(int32_t *tile_total, int64_t n_tiles, int32_t *grand) {
    __shared__ int32_t sw[32];
    int32_t carry = 0;
    for (int64_t b = 0; b < n_tiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int32_t v = i < n_tiles ? tile_total[i] : 0;
        int32_t tot;
        const int32_t ex = block_exclusive_sum(v, sw, tot);
        if (i < n_tiles) tile_total[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *grand = carry;
}

template <class Fn>
__global__ void scan_tile_emit(Fn fn, int64_t n, const int32_t *tile_offset) {
    __shared__ int32_t sw[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = base + j < n ? fn.value(base + j) : 0;
        s += v[j];
    }
    int32_t tot;
    int32_t run = tile_offset[blockIdx.x] + block_exclusive_sum(s, sw, tot);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (base + j < n) fn.emit(base + j, v[j], run);
        run += v[j];
    }
}

// Runs the scan; returns the grand total (synchronises `st`).
template <class Fn>
static int scan_run(Ctx &cx, Fn fn, int64_t n, int64_t *total) {
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 0) {
        *total = 0;
        return 0;
    }
    DevBuf tt, gr;
    if (cx.alloc(tt, tiles * sizeof(int32_t)) || cx.alloc(gr, sizeof(int32_t))) return -1;
    scan_tile_totals<<<(unsigned)tiles, SCAN_THREADS, 0, cx.stream>>>(fn, n, (int32_t *)tt.p);
    scan_tile_offsets<<<1, 1024, 0, cx.stream>>>((int32_t *)tt.p, tiles, (int32_t *)gr.p);
    scan_tile_emit<<<(unsigned)tiles, SCAN_THREADS, 0, cx.stream>>>(fn, n, (const int32_t *)tt.p);
    int32_t h = 0;
    if (cx.check(cudaMemcpyAsync(&h, gr.p, sizeof(int32_t), cudaMemcpyDeviceToHost, cx.stream), "scan total") ||
        cx.check(cudaStreamSynchronize(cx.stream), "scan sync"))
        return -1;
    cx.release(tt);
    cx.release(gr);
    *total = h;
    return 0;
}

// ------------------------------------------------------------- functors
struct FluidCompaction {           // cell order (Sec. 3.1)
    const uint8_t *flags;
    int32_t *cell_id, *cell_voxel;
    __device__ int32_t value(int64_t v) const { return flags[v] == FLAG_FLUID; }
    __device__ void emit(int64_t v, int32_t val, int32_t ex) const {
        cell_id[v] = val ? ex : -1;
        if (val) cell_voxel[ex] = (int32_t)v;
    }
};

// Brick-8 cell order: scan position pos = brick * 512 + local, bricks of
// 8x8x8 voxels in lexicographic brick order, voxels lexicographic inside a
// brick; positions outside the box (partial bricks at the high faces) are
// skipped.
struct BrickCompaction {
    const uint8_t *flags;
    int32_t *cell_id, *cell_voxel;
    int32_t nx, ny, nz, nbx, nby;
    __device__ int64_t voxel(int64_t pos) const {
        const int64_t b = pos >> 9;
        const int l = (int)(pos & 511);
        const int x = (int)(b % nbx) * 8 + (l & 7);
        const int y = (int)((b / nbx) % nby) * 8 + ((l >> 3) & 7);
        const int z = (int)(b / ((int64_t)nbx * nby)) * 8 + (l >> 6);
        if (x >= nx || y >= ny || z >= nz) return -1;
        return x + (int64_t)nx * (y + (int64_t)ny * z);
    }
    __device__ int32_t value(int64_t pos) const {
        const int64_t v = voxel(pos);
        return v >= 0 && flags[v] == FLAG_FLUID;
    }
    __device__ void emit(int64_t pos, int32_t val, int32_t ex) const {
        const int64_t v = voxel(pos);
        if (v < 0) return;
        cell_id[v] = val ? ex : -1;
        if (val) cell_voxel[ex] = (int32_t)v;
    }
};

// Hybrid cell order (SLBM_ORDER_HYBRID): the full bricks first (brick j of
// them holds cells 512 j .. 512 j + 511, voxels lexicographic inside), then
// every other fluid voxel in brick-8 order.  A brick is full when it lies
// wholly inside the box and its 512 voxels are fluid.
__global__ void brick_full_kernel(const uint8_t *flags, int32_t nx, int32_t ny, int32_t nz, int32_t nbx, int32_t nby,
                                  int64_t n_bricks, uint8_t *full) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bricks) return;
    const int x0 = (int)(b % nbx) * 8, y0 = (int)((b / nbx) % nby) * 8, z0 = (int)(b / ((int64_t)nbx * nby)) * 8;
    uint8_t f = x0 + 8 <= nx && y0 + 8 <= ny && z0 + 8 <= nz;
    for (int l = 0; l < 512 && f; ++l) {
        const int64_t v = (x0 + (l & 7)) + (int64_t)nx * ((y0 + ((l >> 3) & 7)) + (int64_t)ny * (z0 + (l >> 6)));
        f = flags[v] == FLAG_FLUID;
    }
    full[b] = f;
}

struct FullBrickScan {             // rank of each full brick among the full ones
    const uint8_t *full;
    int32_t *rank;
    __device__ int32_t value(int64_t b) const { return full[b]; }
    __device__ void emit(int64_t b, int32_t val, int32_t ex) const { rank[b] = val ? ex : -1; }
};

// The fluid voxels of the other bricks, numbered from `base` in brick-8 order.
struct HybridRestCompaction {
    BrickCompaction brick;
    const uint8_t *full;
    int32_t base;
    __device__ int32_t value(int64_t pos) const { return !full[pos >> 9] && brick.value(pos); }
    __device__ void emit(int64_t pos, int32_t val, int32_t ex) const {
        if (full[pos >> 9]) return;
        const int64_t v = brick.voxel(pos);
        if (v < 0) return;
        brick.cell_id[v] = val ? base + ex : -1;
        if (val) brick.cell_voxel[base + ex] = (int32_t)v;
    }
};

// Cells of the full bricks: thread per (brick, local voxel).
__global__ void emit_full_bricks(const int32_t *rank, int32_t nx, int32_t ny, int32_t nbx, int32_t nby,
                                 int64_t n_bricks, int32_t *cell_id, int32_t *cell_voxel) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bricks * 512) return;
    const int64_t b = t >> 9;
    const int32_t r = rank[b];
    if (r < 0) return;
    const int l = (int)(t & 511);
    const int x = (int)(b % nbx) * 8 + (l & 7), y = (int)((b / nbx) % nby) * 8 + ((l >> 3) & 7),
              z = (int)(b / ((int64_t)nbx * nby)) * 8 + (l >> 6);
    const int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
    const int32_t k = r * 512 + l;
    cell_id[v] = k;
    cell_voxel[k] = (int32_t)v;
}

struct InletList {                 // ascending voxel ids of inlet voxels
    const uint8_t *flags;
    int32_t *inlet_voxel;
    __device__ int32_t value(int64_t v) const { return flags[v] == FLAG_INLET; }
    __device__ void emit(int64_t v, int32_t val, int32_t ex) const {
        if (val) inlet_voxel[ex] = (int32_t)v;
    }
};

struct BoundaryCells {             // first link of each cell that has links
    const int32_t *link_cell;
    int32_t *bcell, *bfirst;
    __device__ int32_t value(int64_t b) const { return b == 0 || link_cell[b - 1] != link_cell[b]; }
    __device__ void emit(int64_t b, int32_t val, int32_t ex) const {
        if (val) {
            bcell[ex] = link_cell[b];
            bfirst[ex] = (int32_t)b;
        }
    }
};

// ltile[t] = the first link b with link_cell[b] >= 32 t (link_cell is
// ascending), t = 0 .. n_tiles: thread b fills the tiles after the previous
// link's cell up to its own.
__global__ void link_tiles_kernel(const int32_t *__restrict__ link_cell, int32_t n_links, int32_t n_tiles,
                                  int32_t *__restrict__ ltile) {
    const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > n_links) return;
    const int32_t lo = b == 0 ? 0 : link_cell[b - 1] / EVEN_LINK_TILE + 1;
    const int32_t hi = b == n_links ? n_tiles : link_cell[b] / EVEN_LINK_TILE;
    for (int32_t t = lo; t <= hi; ++t) ltile[t] = b;
}

struct CountScan {                 // exclusive offsets of per-cell link counts
    const uint8_t *count;
    int32_t *offset;
    __device__ int32_t value(int64_t k) const { return count[k]; }
    __device__ void emit(int64_t k, int32_t, int32_t ex) const { offset[k] = ex; }
};

// --------------------------------------------------------- neighbour walk
struct Box {
    int32_t nx, ny, nz;
    uint32_t periodic;
};

// Voxel at x - c_i (the pull neighbour of direction i), or -1 when it lies
// outside the box across a non-periodic face (treated as a wall).
template <int Q>
__device__ __forceinline__ int64_t pull_neighbour(const Box &b, int x, int y, int z, int i) {
    int nx = x - cx(i), ny = y - cy(i), nz = z - cz(i);
    if (nx < 0 || nx >= b.nx) {
        if (!(b.periodic & 1u)) return -1;
        nx = (nx + b.nx) % b.nx;
    }
    if (ny < 0 || ny >= b.ny) {
        if (!(b.periodic & 2u)) return -1;
        ny = (ny + b.ny) % b.ny;
    }
    if (nz < 0 || nz >= b.nz) {
        if (!(b.periodic & 4u)) return -1;
        nz = (nz + b.nz) % b.nz;
    }
    return (int64_t)nx + (int64_t)b.nx * ((int64_t)ny + (int64_t)b.ny * nz);
}

__device__ __forceinline__ void voxel_xyz(const Box &b, int64_t v, int &x, int &y, int &z) {
    x = (int)(v % b.nx);
    const int64_t r = v / b.nx;
    y = (int)(r % b.ny);
    z = (int)(r / b.ny);
}

template <int Q>
__global__ void count_links(Box b, const uint8_t *flags, const int32_t *cell_voxel, int32_t nf,
                            uint8_t *count) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    int x, y, z;
    voxel_xyz(b, cell_voxel[k], x, y, z);
    int c = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int64_t nb = pull_neighbour<Q>(b, x, y, z, i);
        const uint8_t t = nb < 0 ? (uint8_t)FLAG_WALL : flags[nb];
        c += (t == FLAG_INLET || t == FLAG_OUTLET);
    }
    count[k] = (uint8_t)c;
}

// Index of voxel v in the sorted inlet list (binary search), or -1.
__device__ __forceinline__ int64_t inlet_rank(const int32_t *list, int64_t n, int64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (list[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && list[lo] == v) ? lo : -1;
}

// One thread per cell; writes its Q-1 entries (column k of each row) and its
// boundary links.  The canonical pull entry P(i,k) (Sec. 3.1: fluid
// neighbour -> i*S + n, wall -> inverse(i)*S + k, inlet/outlet -> -(b+1)) is
// stored in the form the AA odd step reads: non-negative entries with their
// row flipped (flip_row), i.e. the odd-step slot R(i,k).  The flip is exact
// and its own inverse; sparse_lbm_export_lists flips back to P.  Link maps are
// in shifted, unscaled units.
template <int Q>
__global__ void build_index(Box b, const uint8_t *flags, const int32_t *cell_id,
                            const int32_t *cell_voxel, int32_t nf, int32_t S, int32_t *P,
                            const int32_t *link_offset, int32_t *link_cell, int32_t *link_dir,
                            int32_t *link_type, LinkMap *maps, const int32_t *inlet_voxel,
                            int64_t n_inlet, const float *inlet_u, float rho_out) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    if (k >= nf) {
#pragma unroll
        for (int i = 1; i < Q; ++i) P[(int64_t)(i - 1) * S + k] = INT32_MIN;
        return;
    }
    int x, y, z;
    voxel_xyz(b, cell_voxel[k], x, y, z);
    int32_t nb_link = link_offset ? link_offset[k] : 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int64_t nb = pull_neighbour<Q>(b, x, y, z, i);
        const uint8_t t = nb < 0 ? (uint8_t)FLAG_WALL : flags[nb];
        int32_t e;
        if (t == FLAG_FLUID) {
            e = i * S + cell_id[nb];
        } else if (t == FLAG_WALL) {
            e = inv(i) * S + k;
        } else {
            const int32_t l = nb_link++;
            e = -(l + 1);
            link_cell[l] = k;
            link_dir[l] = i;
            link_type[l] = t;
            LinkMap m;
            m.cx = (float)cx(i);
            m.cy = (float)cy(i);
            m.cz = (float)cz(i);
            if (t == FLAG_INLET) {
                float ux = 0.f, uy = 0.f, uz = 0.f;
                if (inlet_u) {
                    const int64_t r = inlet_rank(inlet_voxel, n_inlet, nb);
                    if (r >= 0) {
                        ux = inlet_u[3 * r];
                        uy = inlet_u[3 * r + 1];
                        uz = inlet_u[3 * r + 2];
                    }
                }
                m.s = 1.0f;
                m.a = 6.0f * wgt<Q>(i) * (cx(i) * ux + cy(i) * uy + cz(i) * uz);
                m.q2 = 0.0f;
            } else {
                m.s = -1.0f;
                m.a = 2.0f * wgt<Q>(i) * (rho_out - 1.0f);
                m.q2 = 2.0f * wgt<Q>(i) * rho_out;
            }
            maps[l] = m;
        }
        P[(int64_t)(i - 1) * S + k] = e >= 0 ? flip_row(e, i, S) : e;
    }
}

// Odd-step slots -> canonical pull entries (the inverse of the flip above),
// into a separate buffer for export.
__global__ void unflip_rows(const int32_t *R, int32_t S, int32_t rows, int32_t *P) {
    const int64_t n = (int64_t)rows * S;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = R[j];
        const int i = (int)(j / S) + 1;
        P[j] = e >= 0 ? flip_row(e, i, S) : e;
    }
}

cudaError_t launch_unflip(const Domain &d, int32_t *out, cudaStream_t st) {
    const int64_t n = (int64_t)(d.q - 1) * d.S;
    if (n == 0) return cudaSuccess;
    unflip_rows<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, st>>>(
        (const int32_t *)d.P.p, (int32_t)d.S, d.q - 1, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- driver
int build_sparse_lists(Ctx &cx, Domain &d, const uint8_t *d_flags, bool has_bc, const float *h_inlet_u,
                       int64_t n_inlet_u) {
    const int64_t N = d.n_vox;
    Box b{d.nx, d.ny, d.nz, d.periodic};
    DevBuf cell_id;
    if (cx.alloc(cell_id, N * sizeof(int32_t)) || cx.alloc(d.cell_voxel, std::max<int64_t>(N, 1) * sizeof(int32_t)))
        return -1;
    int64_t nf = 0;
    if (d.order == SLBM_ORDER_BRICK8) {
        const int32_t nbx = (d.nx + 7) / 8, nby = (d.ny + 7) / 8, nbz = (d.nz + 7) / 8;
        const int64_t positions = (int64_t)nbx * nby * nbz * 512;
        if (scan_run(cx, BrickCompaction{d_flags, (int32_t *)cell_id.p, (int32_t *)d.cell_voxel.p, d.nx, d.ny, d.nz,
                                         nbx, nby},
                     positions, &nf))
            return -1;
    } else if (d.order == SLBM_ORDER_HYBRID) {
        const int32_t nbx = (d.nx + 7) / 8, nby = (d.ny + 7) / 8, nbz = (d.nz + 7) / 8;
        const int64_t n_bricks = (int64_t)nbx * nby * nbz;
        DevBuf full, rank;
        if (cx.alloc(full, n_bricks) || cx.alloc(rank, n_bricks * sizeof(int32_t))) return -1;
        brick_full_kernel<<<(unsigned)((n_bricks + 127) / 128), 128, 0, cx.stream>>>(
            d_flags, d.nx, d.ny, d.nz, nbx, nby, n_bricks, (uint8_t *)full.p);
        int64_t n_full = 0, rest = 0;
        if (cx.check(cudaGetLastError(), "brick_full launch") ||
            scan_run(cx, FullBrickScan{(const uint8_t *)full.p, (int32_t *)rank.p}, n_bricks, &n_full))
            return -1;
        if (n_full > 0) {
            emit_full_bricks<<<(unsigned)((n_bricks * 512 + 255) / 256), 256, 0, cx.stream>>>(
                (const int32_t *)rank.p, d.nx, d.ny, nbx, nby, n_bricks, (int32_t *)cell_id.p,
                (int32_t *)d.cell_voxel.p);
            if (cx.check(cudaGetLastError(), "emit_full_bricks launch")) return -1;
        }
        const BrickCompaction bc{d_flags, (int32_t *)cell_id.p, (int32_t *)d.cell_voxel.p, d.nx, d.ny, d.nz, nbx, nby};
        if (scan_run(cx, HybridRestCompaction{bc, (const uint8_t *)full.p, (int32_t)(n_full * 512)}, n_bricks * 512,
                     &rest))
            return -1;
        cx.release(full);
        cx.release(rank);
        d.n_full_cells = n_full * 512;
        nf = d.n_full_cells + rest;
    } else if (scan_run(cx, FluidCompaction{d_flags, (int32_t *)cell_id.p, (int32_t *)d.cell_voxel.p}, N, &nf)) {
        return -1;
    }
    d.n_fluid = nf;
    d.S = (nf + 127) / 128 * 128;
    if ((int64_t)d.q * d.S >= ((int64_t)1 << 31)) {
        cx.fail(SLBM_EUNSUPPORTED, "Q * stride >= 2^31: domain too large for int32 slots");
        return -1;
    }
    // shrink cell_voxel to N_F entries
    if (nf < N) {
        DevBuf cv;
        if (cx.alloc(cv, std::max<int64_t>(nf, 1) * sizeof(int32_t))) return -1;
        if (nf && cx.check(cudaMemcpyAsync(cv.p, d.cell_voxel.p, nf * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                           cx.stream), "copy cell_voxel"))
            return -1;
        cx.release(d.cell_voxel);
        d.cell_voxel = cv;
        cv.p = nullptr;
    }
    if (d.S == 0) {
        cx.release(cell_id);
        return 0;
    }
    if (cx.alloc(d.P, (int64_t)(d.q - 1) * d.S * sizeof(int32_t))) return -1;

    DevBuf link_count, link_offset, inlet_voxel, inlet_u;
    int64_t n_links = 0, n_inlet = 0;
    if (has_bc) {
        if (cx.alloc(link_count, nf)) return -1;
        const unsigned gb = (unsigned)((nf + 255) / 256);
        if (d.q == 19)
            count_links<19><<<gb, 256, 0, cx.stream>>>(b, d_flags, (int32_t *)d.cell_voxel.p, (int32_t)nf,
                                                       (uint8_t *)link_count.p);
        else
            count_links<27><<<gb, 256, 0, cx.stream>>>(b, d_flags, (int32_t *)d.cell_voxel.p, (int32_t)nf,
                                                       (uint8_t *)link_count.p);
        if (cx.alloc(link_offset, nf * sizeof(int32_t))) return -1;
        if (scan_run(cx, CountScan{(const uint8_t *)link_count.p, (int32_t *)link_offset.p}, nf, &n_links)) return -1;
        cx.release(link_count);
        d.n_links = n_links;
        if (n_links) {
            if (cx.alloc(d.link_cell, n_links * 4) || cx.alloc(d.link_dir, n_links * 4) ||
                cx.alloc(d.link_type, n_links * 4) || cx.alloc(d.link_map, n_links * sizeof(LinkMap)))
                return -1;
        }
        if (h_inlet_u) {
            if (cx.alloc(inlet_voxel, std::max<int64_t>(n_inlet_u, 1) * sizeof(int32_t))) return -1;
            if (scan_run(cx, InletList{d_flags, (int32_t *)inlet_voxel.p}, N, &n_inlet)) return -1;
            if (n_inlet != n_inlet_u) {
                cx.fail(SLBM_EINVAL, "n_inlet_u does not match the number of inlet voxels");
                return -1;
            }
            if (cx.alloc(inlet_u, std::max<int64_t>(n_inlet, 1) * 3 * sizeof(float))) return -1;
            if (n_inlet && cx.check(cudaMemcpyAsync(inlet_u.p, h_inlet_u, n_inlet * 3 * sizeof(float),
                                                    cudaMemcpyHostToDevice, cx.stream), "inlet_u H2D"))
                return -1;
        }
    }
    const unsigned gs = (unsigned)((d.S + 255) / 256);
    auto launch = [&](auto qtag) {
        constexpr int QQ = decltype(qtag)::value;
        build_index<QQ><<<gs, 256, 0, cx.stream>>>(
            b, d_flags, (const int32_t *)cell_id.p, (const int32_t *)d.cell_voxel.p, (int32_t)nf, (int32_t)d.S,
            (int32_t *)d.P.p, has_bc ? (const int32_t *)link_offset.p : nullptr, (int32_t *)d.link_cell.p,
            (int32_t *)d.link_dir.p, (int32_t *)d.link_type.p, (LinkMap *)d.link_map.p,
            (const int32_t *)inlet_voxel.p, n_inlet, (const float *)inlet_u.p, (float)d.rho_out);
    };
    if (d.q == 19) launch(std::integral_constant<int, 19>{});
    else launch(std::integral_constant<int, 27>{});
    if (cx.check(cudaGetLastError(), "build_index launch") || cx.check(cudaStreamSynchronize(cx.stream), "build sync"))
        return -1;
    if (d.order == SLBM_ORDER_HYBRID && d.layout == SLBM_LAYOUT_SPARSE && d.n_full_cells > 0) {   // face lists
        const int64_t entries = d.n_full_cells / 512 * (d.q == 19 ? face_block<19>() : face_block<27>());
        if (cx.alloc(d.face, entries * sizeof(int32_t))) return -1;
        const unsigned gf = (unsigned)((d.n_full_cells + 255) / 256);
        if (d.q == 19)
            build_face_list<19><<<gf, 256, 0, cx.stream>>>((const int32_t *)d.P.p, (int32_t)d.S,
                                                           (int32_t)d.n_full_cells, (int32_t *)d.face.p);
        else
            build_face_list<27><<<gf, 256, 0, cx.stream>>>((const int32_t *)d.P.p, (int32_t)d.S,
                                                           (int32_t)d.n_full_cells, (int32_t *)d.face.p);
        if (cx.check(cudaGetLastError(), "build_face_list launch")) return -1;
    }
    if (n_links > 0) {   // cells with links, for the fix-up around the even step
        if (cx.alloc(d.bcell, n_links * 4) || cx.alloc(d.bfirst, (n_links + 1) * 4)) return -1;
        int64_t nb = 0;
        if (scan_run(cx, BoundaryCells{(const int32_t *)d.link_cell.p, (int32_t *)d.bcell.p, (int32_t *)d.bfirst.p},
                     n_links, &nb))
            return -1;
        d.n_bcells = nb;
        const int32_t end = (int32_t)n_links;
        if (cx.check(cudaMemcpyAsync((int32_t *)d.bfirst.p + nb, &end, 4, cudaMemcpyHostToDevice, cx.stream),
                     "bfirst end") ||
            cx.alloc(d.bc_ubuf, nb * 3 * sizeof(float)))
            return -1;
        // first link of each 32-cell tile, for the even kernels that apply
        // the link maps themselves
        const int32_t n_tiles = (int32_t)((d.n_fluid + EVEN_LINK_TILE - 1) / EVEN_LINK_TILE);
        if (cx.alloc(d.ltile, ((int64_t)n_tiles + 1) * 4)) return -1;
        link_tiles_kernel<<<(unsigned)((n_links + 1 + 255) / 256), 256, 0, cx.stream>>>(
            (const int32_t *)d.link_cell.p, (int32_t)n_links, n_tiles, (int32_t *)d.ltile.p);
        if (cx.check(cudaGetLastError(), "link_tiles launch") ||
            cx.check(cudaStreamSynchronize(cx.stream), "boundary cells"))
            return -1;
    }
    cx.release(cell_id);
    cx.release(link_offset);
    cx.release(inlet_voxel);
    cx.release(inlet_u);
    return 0;
}

// ------------------------------------------------------------- link codes
// 16-bit form of the odd-step slots R(i, k).  A fluid neighbour's slot lies in
// row inverse(i), so only its column needs storing; within a tile of
// CODE_TILE consecutive cells the columns of one direction span little more
// than the tile (neighbours of consecutive cells are near-consecutive in the
// compacted order), so they are stored relative to the tile's smallest one:
//   code = column - base       fluid neighbour
//   code = CODE_WALL           wall: the cell's own slot i*S + k (and padding)
//   code = CODE_ESCAPE         inlet/outlet link: read R(i, k) itself
// base[tile * (Q-1) + i-1] is the smallest fluid column (0 if none), or -1
// when the tile-direction's columns span CODE_ESCAPE or more (e.g. across a
// periodic wrap): then every slot of the tile-direction is read from R
// itself and its codes are CODE_ESCAPE.  One CTA per tile; the span is
// reduced in a fixed order, so the codes are deterministic.
template <int Q>
__global__ void __launch_bounds__(CODE_TILE) build_codes_kernel(const int32_t *__restrict__ R, int32_t S, int32_t nf,
                                                                uint16_t *__restrict__ code,
                                                                int32_t *__restrict__ base) {
    constexpr int W = CODE_TILE / 32;
    __shared__ int32_t wlo[W], whi[W];
    const int32_t k = blockIdx.x * CODE_TILE + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 1; i < Q; ++i) {
        const int32_t e = k < nf ? R[(i - 1) * S + k] : 0;
        const bool link = k < nf && e < 0;                    // inlet/outlet
        const bool fluid = k < nf && e >= 0 && e / S != i;    // row inverse(i)
        const int32_t col = fluid ? e - inv(i) * S : 0;
        int32_t lo = fluid ? col : INT32_MAX, hi = fluid ? col : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            wlo[warp] = lo;
            whi[warp] = hi;
        }
        __syncthreads();
        lo = wlo[0];
        hi = whi[0];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            lo = min(lo, wlo[w]);
            hi = max(hi, whi[w]);
        }
        __syncthreads();                                  // wlo/whi are reused by the next direction
        const bool wide = hi >= 0 && hi - lo >= (int32_t)CODE_ESCAPE;
        const int32_t b = wide ? -1 : (hi < 0 ? 0 : lo);
        uint16_t c = (uint16_t)CODE_WALL;                 // walls and padding
        if (wide || link) c = (uint16_t)CODE_ESCAPE;
        else if (fluid) c = (uint16_t)(col - b);          // below CODE_ESCAPE
        code[(int64_t)(i - 1) * S + k] = c;
        if (threadIdx.x == 0) base[(int64_t)blockIdx.x * (Q - 1) + (i - 1)] = b;
    }
}

int build_link_codes(Ctx &cx, Domain &d) {
    if (d.S == 0) return 0;
    const int64_t tiles = d.S / CODE_TILE;
    if (cx.alloc(d.code, (int64_t)(d.q - 1) * d.S * sizeof(uint16_t)) ||
        cx.alloc(d.code_base, tiles * (d.q - 1) * sizeof(int32_t)))
        return -1;
    if (d.q == 19)
        build_codes_kernel<19><<<(unsigned)tiles, CODE_TILE, 0, cx.stream>>>(
            (const int32_t *)d.P.p, (int32_t)d.S, (int32_t)d.n_fluid, (uint16_t *)d.code.p, (int32_t *)d.code_base.p);
    else
        build_codes_kernel<27><<<(unsigned)tiles, CODE_TILE, 0, cx.stream>>>(
            (const int32_t *)d.P.p, (int32_t)d.S, (int32_t)d.n_fluid, (uint16_t *)d.code.p, (int32_t *)d.code_base.p);
    return cx.check(cudaGetLastError(), "build_codes launch");
}

int build_window_tab(Ctx &cx, Domain &d) {
    if (d.S == 0) return 0;
    const int64_t n = d.S / WIN_TILE * (d.q - 1);
    if (cx.alloc(d.win_tab, n * (int64_t)sizeof(WinSpan)) ||
        cx.alloc(d.win_code, (int64_t)(d.q - 1) * d.S * (int64_t)sizeof(uint16_t)))
        return -1;
    const unsigned grid = (unsigned)((n + 127) / 128);
    const dim3 cgrid((unsigned)((d.S + 255) / 256), (unsigned)(d.q - 1));
    const int32_t *R = (const int32_t *)d.P.p;
    WinSpan *tab = (WinSpan *)d.win_tab.p;
    uint16_t *code = (uint16_t *)d.win_code.p;
    if (d.q == 19) {
        build_window_table<19><<<grid, 128, 0, cx.stream>>>(R, (int32_t)d.S, (int32_t)d.n_fluid, tab);
        build_window_codes<19><<<cgrid, 256, 0, cx.stream>>>(R, (int32_t)d.S, (int32_t)d.n_fluid, tab, code);
    } else {
        build_window_table<27><<<grid, 128, 0, cx.stream>>>(R, (int32_t)d.S, (int32_t)d.n_fluid, tab);
        build_window_codes<27><<<cgrid, 256, 0, cx.stream>>>(R, (int32_t)d.S, (int32_t)d.n_fluid, tab, code);
    }
    return cx.check(cudaGetLastError(), "build_window_table launch");
}

}  // namespace slbm

// ------------------------------------------------ allocation-free compaction
// sparse_lbm_compact_noalloc: the same three-phase compaction scan, with the
// per-tile totals kept in a fixed device array that lives as long as the
// library stays loaded, instead of in memory allocated per call.
#include <mutex>

namespace slbm {

constexpr int64_t NOALLOC_MAX_TILES = 65536;   // SLBM_NOALLOC_MAX_VOXELS / SCAN_TILE
static_assert(NOALLOC_MAX_TILES * SCAN_TILE == SLBM_NOALLOC_MAX_VOXELS, "limit mismatch");

// Tile totals of the scan (256 KiB).  Every call overwrites the entries it
// uses before reading them, so nothing needs clearing between calls.
static __device__ __align__(256) int32_t g_noalloc_tiles[NOALLOC_MAX_TILES];

// Device address of g_noalloc_tiles per device.  The host-side name of the
// array is not a device address, so every call made outside a stream capture
// looks the address up with its device current (a device reset that reloads
// the module moves the array); a call inside a capture, where the lookup is
// not allowed, uses the address the last call outside capture found.
static std::mutex g_noalloc_mu;
static int32_t *g_noalloc_addr[128] = {};

static int noalloc_scratch(cudaStream_t st, int32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        set_error(SLBM_ECUDA, "sparse_lbm_compact_noalloc: no current CUDA device");
        return -1;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(SLBM_ECUDA, std::string("sparse_lbm_compact_noalloc: cudaStreamIsCapturing: ") +
                                  cudaGetErrorString(e));
        return -1;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_tiles);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error(SLBM_ECUDA, std::string("sparse_lbm_compact_noalloc: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
            return -1;
        }
        g_noalloc_addr[dev] = (int32_t *)p;
    } else if (!g_noalloc_addr[dev]) {
        set_error(SLBM_ECUDA, "sparse_lbm_compact_noalloc: first call on this device made during a stream "
                              "capture (call it once outside capture first)");
        return -1;
    }
    *out = g_noalloc_addr[dev];
    return 0;
}

}  // namespace slbm

extern "C" slbm_status sparse_lbm_compact_noalloc(const uint8_t *flags, int64_t n_voxels, int32_t *cell_id,
                                                  int32_t *cell_voxel, int32_t *n_fluid, void *stream) {
    using namespace slbm;
    if (n_voxels < 0 || n_voxels > SLBM_NOALLOC_MAX_VOXELS) {
        set_error(SLBM_EINVAL, "sparse_lbm_compact_noalloc: n_voxels must lie in [0, SLBM_NOALLOC_MAX_VOXELS = "
                               "268435456]");
        return SLBM_EINVAL;
    }
    if (!n_fluid || (n_voxels > 0 && (!flags || !cell_id || !cell_voxel))) {
        set_error(SLBM_EINVAL, "sparse_lbm_compact_noalloc: null device pointer");
        return SLBM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *tiles = nullptr;
    if (noalloc_scratch(st, &tiles)) return SLBM_ECUDA;
    cudaError_t e;
    if (n_voxels == 0) {
        e = cudaMemsetAsync(n_fluid, 0, sizeof(int32_t), st);
    } else {
        const int64_t nt = (n_voxels + SCAN_TILE - 1) / SCAN_TILE;
        const FluidCompaction fn{flags, cell_id, cell_voxel};
        scan_tile_totals<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(fn, n_voxels, tiles);
        scan_tile_offsets<<<1, 1024, 0, st>>>(tiles, nt, n_fluid);
        scan_tile_emit<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(fn, n_voxels, tiles);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(SLBM_ECUDA, std::string("sparse_lbm_compact_noalloc: ") + cudaGetErrorString(e));
        return SLBM_ECUDA;
    }
    set_error(SLBM_OK, "");
    return SLBM_OK;
}
