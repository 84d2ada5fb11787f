// aa_window.cuh -- the AA odd step (Sec. 5.1) with every read of a tile of
// cells staged in shared memory by the bulk-copy engine (launch variant 6).
//
// In the plain odd kernel each cell first loads its Q-1 slots R(i,k) from
// the index-list and only then gathers the populations they point at: two
// dependent trips to DRAM per cell, and the kernel waits on memory latency
// (registers limit the warps that keep loads in flight).  Here the reads of
// a tile are known before its threads run:
//   - the tile's Q-1 index-list rows (R(i,k) for its 128 cells);
//   - its own Q rows of the PDF-list (a wall or boundary link of direction i
//     reads the cell's own slot in row i, and the rest population row 0);
//   - per direction i, a window of row inverse(i): with cells numbered
//     lexicographically, the pull neighbours x_k - c_i of 128 consecutive
//     cells have column ids k + delta_i(k) with a nearly constant offset, so
//     a window of the tile's width plus a margin holds almost every fluid
//     neighbour's slot (a neighbour across a periodic wrap falls outside and
//     is read from global memory).
// A per-tile table (built once per domain, `build_window_table`) gives each
// window's first column and length; it is copied in with the tile.  Instead
// of the tile's int32 index rows, the stage holds 16-bit window codes (built
// with the table, `build_window_codes`): per link, the position of the slot
// R(i,k) among the stage's staged populations (own rows, then windows), or an
// escape value for a fluid neighbour outside its window and for a boundary
// link, which read the int32 slot list instead.  A cell then gathers with one
// shared-memory load per link, recovers R(i,k) for the scatter from the code
// and its window's first column, and the odd step reads 2 index bytes per
// link instead of 4.  One warp issues the copies of tile t + NSTAGE*grid
// into a ring of NSTAGE stages while the other warps compute tile t from
// shared memory, so the copy engine keeps the DRAM reads in flight and the
// computing threads only compute and scatter.  The scatter to the slots read
// stays a plain store per population.
//
// Reading the windows in place is race-free: each slot is read and written
// by one cell only (the AA odd step writes back to the slots it read), so
// the other cells' values that a window copy may catch before or after their
// update are never used.
#pragma once

#include "aa_kernels.cuh"

namespace slbm {

constexpr int WIN_TILE = 128;                 // cells per tile (= threads per CTA)
constexpr int WIN_MARGIN = 16;                // cells of slack on each side of a window
constexpr int WIN_CELLS = WIN_TILE + 2 * WIN_MARGIN + 8;   // main window capacity (alignment included)
constexpr int WIN2_CELLS = 24;                // secondary window capacity

// Table entry of one tile and direction: the main window (first column in
// row inverse(i), a multiple of 8, and length in cells, a multiple of 8; 0 =
// no fluid neighbour in that direction) and a short secondary window for the
// fluid neighbours the main one misses -- with lexicographic numbering these
// are the pull neighbours across the periodic x wrap, at the far end of the
// same row (0 = none, or they do not fit).
struct WinSpan {
    int32_t first, len, first2, len2;
};

// Codes: bits 0-14 a position among the staged populations, bit 15 set for
// a boundary link (gather from the own slot, scatter through the link map);
// WIN_ESCAPE: a fluid neighbour outside both windows (read through the int32
// slot list).
constexpr uint32_t WIN_ESCAPE = 0xFFFF;
constexpr uint32_t WIN_LINK = 0x8000;

// Byte layout of one stage of the ring, for Q directions and element type T:
// the codes, the staged populations (own rows [Q][TILE], main windows
// [Q-1][WIN_CELLS], secondary windows [Q-1][WIN2_CELLS]) and the table.
template <int Q, class T>
struct WinStage {
    static constexpr int R1 = Q - 1;
    static constexpr uint32_t OWN_ELEMS = Q * WIN_TILE;                        // code < OWN_ELEMS: own slot
    static constexpr uint32_t WIN2_ELEMS = OWN_ELEMS + R1 * WIN_CELLS;         // first secondary position
    static constexpr uint32_t POP_ELEMS = WIN2_ELEMS + R1 * WIN2_CELLS;
    static constexpr uint32_t CODE = 0;                                        // uint16 [R1][TILE]
    static constexpr uint32_t POP = CODE + R1 * WIN_TILE * 2;                  // T [POP_ELEMS]
    static constexpr uint32_t TAB = POP + ((POP_ELEMS * sizeof(T) + 15) / 16) * 16;
    static constexpr uint32_t BYTES = TAB + ((R1 * sizeof(WinSpan) + 15) / 16) * 16;
    static_assert(POP_ELEMS < WIN_LINK, "positions fit in 15 bits");
};

// Window table of one domain: for tile t and direction i = r + 1, the fluid
// neighbours' columns n (slot R(i,k) = inverse(i)*S + n) of the tile's cells.
// The main window is centred on the offset n - k of one of three reference
// cells (the first, middle and last fluid-linked cell of the tile), whichever
// covers most of the tile's links, with WIN_MARGIN cells of slack, clipped to
// [0, S); the secondary one spans the remaining columns if they lie within
// WIN2_CELLS of each other.  One thread per (tile, direction).
template <int Q>
__global__ void build_window_table(const int32_t *__restrict__ R, int32_t S, int32_t nf, WinSpan *__restrict__ tab) {
    const int32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t tiles = S / WIN_TILE;
    if (id >= tiles * (Q - 1)) return;
    const int32_t t = id / (Q - 1), r = id % (Q - 1);
    const int ib = inv(r + 1);
    const int64_t row0 = (int64_t)ib * S;
    const int32_t k0 = t * WIN_TILE;
    const int32_t kend = min(nf, k0 + WIN_TILE);
    auto offset_of = [&](int32_t k) -> int64_t {        // n - k of a fluid link, or a sentinel
        const int32_t e = R[(int64_t)r * S + k];
        return (e >= row0 && e < row0 + S) ? (int64_t)e - row0 - k : INT64_MIN;
    };
    int32_t first = -1, last = -1, mid = -1, mid_d = 1 << 30;
    for (int32_t k = k0; k < kend; ++k) {
        if (offset_of(k) == INT64_MIN) continue;
        if (first < 0) first = k;
        last = k;
        const int32_t dm = abs(k - (k0 + WIN_TILE / 2));
        if (dm < mid_d) {
            mid_d = dm;
            mid = k;
        }
    }
    WinSpan w{0, 0, 0, 0};
    if (first >= 0) {
        const int32_t refs[3] = {first, mid, last};
        int32_t best = -1;
        for (int c = 0; c < 3; ++c) {
            const int64_t d = offset_of(refs[c]);
            int64_t lo = (int64_t)k0 + d - WIN_MARGIN;
            lo = lo < 0 ? 0 : (lo / 8) * 8;
            int64_t len = WIN_CELLS;
            if (lo + len > S) lo = S - len;
            if (lo < 0) {
                lo = 0;
                len = S;
            }
            int32_t cov = 0;
            for (int32_t k = k0; k < kend; ++k) {
                const int64_t dk = offset_of(k);
                if (dk == INT64_MIN) continue;
                const int64_t n = k + dk;
                cov += n >= lo && n < lo + len;
            }
            if (cov > best) {
                best = cov;
                w.first = (int32_t)lo;
                w.len = (int32_t)len;
            }
        }
        // the columns the main window misses
        int64_t lo2 = INT64_MAX, hi2 = -1;
        for (int32_t k = k0; k < kend; ++k) {
            const int64_t dk = offset_of(k);
            if (dk == INT64_MIN) continue;
            const int64_t n = k + dk;
            if (n >= w.first && n < w.first + w.len) continue;
            lo2 = n < lo2 ? n : lo2;
            hi2 = n > hi2 ? n : hi2;
        }
        if (hi2 >= 0) {
            lo2 = (lo2 / 8) * 8;
            const int64_t len2 = ((hi2 + 1 - lo2 + 7) / 8) * 8;
            if (len2 <= WIN2_CELLS && lo2 + len2 <= S) {
                w.first2 = (int32_t)lo2;
                w.len2 = (int32_t)len2;
            }
        }
    }
    tab[id] = w;
}

// Window codes of one domain (after the table): per direction i = r + 1 and
// cell k, the position of the slot R(i,k) among the staged populations of
// k's tile -- a fluid neighbour inside its main window: OWN_ELEMS +
// r*WIN_CELLS + (n - first); inside its secondary window: WIN2_ELEMS +
// r*WIN2_CELLS + (n - first2); a wall (R = i*S + k): i*TILE + k mod TILE; a
// boundary link: the same own position with WIN_LINK set -- or WIN_ESCAPE (a
// fluid neighbour outside both windows, padding).
template <int Q>
__global__ void build_window_codes(const int32_t *__restrict__ R, int32_t S, int32_t nf,
                                   const WinSpan *__restrict__ tab, uint16_t *__restrict__ code) {
    using L = WinStage<Q, float>;                      // positions do not depend on the element type
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (k >= S) return;
    const int i = r + 1;
    uint32_t c = WIN_ESCAPE;
    if (k < nf) {
        const int32_t e = R[(int64_t)r * S + k];
        const int32_t row_b = inv(i) * S;
        if (e < 0) {
            c = (i * WIN_TILE + k % WIN_TILE) | WIN_LINK;
        } else if (e - row_b >= 0 && e - row_b < S) {
            const WinSpan w = tab[(int64_t)(k / WIN_TILE) * (Q - 1) + r];
            const int32_t n = e - row_b;
            if (n >= w.first && n < w.first + w.len) c = L::OWN_ELEMS + r * WIN_CELLS + (n - w.first);
            else if (n >= w.first2 && n < w.first2 + w.len2) c = L::WIN2_ELEMS + r * WIN2_CELLS + (n - w.first2);
        } else if (e == i * S + k) {
            c = i * WIN_TILE + k % WIN_TILE;
        }
    }
    code[(int64_t)r * S + k] = (uint16_t)c;
}

// The odd step of one tile's cells from a filled stage.
template <int Q, int ST, bool HAS_BC>
__device__ __forceinline__ void window_cell(typename Store<ST>::T *__restrict__ pdf, const int32_t *__restrict__ R,
                                            const unsigned char *stage, int tid, int32_t k, int32_t S,
                                            const LinkMap *__restrict__ maps, const CollideParams &p) {
    using St = Store<ST>;
    using T = typename St::T;
    using L = WinStage<Q, T>;
    const uint16_t *code = reinterpret_cast<const uint16_t *>(stage + L::CODE);
    const T *pop = reinterpret_cast<const T *>(stage + L::POP);
    const WinSpan *tab = reinterpret_cast<const WinSpan *>(stage + L::TAB);
    float g[Q];
    int32_t slot[Q];
    g[0] = St::raw(pop[tid]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const uint32_t c = code[(i - 1) * WIN_TILE + tid];
        if (c != WIN_ESCAPE) {
            const uint32_t pc = c & (WIN_LINK - 1);
            g[i] = St::raw(pop[pc]);
            // staged position -> slot: own row i, or column first(2) + offset of row inverse(i)
            const WinSpan w = tab[i - 1];
            const int32_t rb = inv(i) * S;
            const int32_t s1 = rb + w.first - (int32_t)L::OWN_ELEMS - (i - 1) * WIN_CELLS + (int32_t)pc;
            const int32_t s2 = rb + w.first2 - (int32_t)L::WIN2_ELEMS - (i - 1) * WIN2_CELLS + (int32_t)pc;
            slot[i] = pc < L::OWN_ELEMS ? i * S + k : (pc < L::WIN2_ELEMS ? s1 : s2);
            // a boundary link's negative entry (its map), loaded while the cell collides
            if (HAS_BC && (c & WIN_LINK)) slot[i] = R[(int64_t)(i - 1) * S + k];
        } else {                                        // a fluid neighbour outside both windows
            const int32_t e = R[(int64_t)(i - 1) * S + k];
            slot[i] = e;
            g[i] = St::raw(__ldg(pdf + e));
        }
    }
    const Vel u = collide<Q, St::scaled>(g, p);
    pdf[k] = St::pack(g[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        float v = g[inv(i)];
        int32_t r = slot[i];
        if (HAS_BC && r < 0) {
            v = apply_link(maps[-(r + 1)], v, u.x, u.y, u.z, p.scale);
            r = i * S + k;
        }
        pdf[r] = St::pack(v);
    }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait on an mbarrier phase that also gives up when another warp of
// the CTA has raised `stop` (time limit ~2^31 SM cycles, about a second).
// Each test lets the hardware suspend the warp for up to ~2 us until the
// phase completes, so a waiting warp takes almost no issue slots.
__device__ __forceinline__ bool mbar_wait_or_stop(uint64_t *bar, uint32_t phase, volatile int32_t *stop) {
    if (mbar_try_wait_suspend(bar, phase)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_suspend(bar, phase)) {
        if (*stop || clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

template <int Q, int ST>
constexpr size_t window_smem_bytes(int nstage) {
    return (size_t)nstage * WinStage<Q, typename Store<ST>::T>::BYTES + (size_t)2 * nstage * sizeof(uint64_t) + 16;
}

// Warp-specialised persistent CTAs: warps 0-3 compute one cell each of a
// WIN_TILE-cell tile, warp 4 only issues the copies.  Tile t of CTA b is b,
// b + grid, ...; its reads go to stage (j mod NSTAGE) of a ring in dynamic
// shared memory (j = the CTA's tile count).  Stage s has a "full" mbarrier
// (one arrival with the transaction bytes; the copies complete it) and an
// "empty" one (the 128 compute threads arrive when done with the stage), so
// the producer runs up to NSTAGE tiles ahead and the compute warps never
// wait for copies to be issued.  Producer lanes copy in parallel: lane r the
// index row r, own row r and window r; lane 0 also own row Q-1 and the
// table entries.  Every wait is bounded; a timeout latches
// ERR_STAGE_TIMEOUT, raises a shared stop word that ends the other warps'
// waits, and the producer waits (bounded) for the copies it still has in
// flight before the CTA exits.
template <int Q, int ST, bool HAS_BC, int NSTAGE>
__global__ void __launch_bounds__(WIN_TILE + 32) aa_odd_window_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                                      const int32_t *__restrict__ R, int32_t S,
                                                                      int32_t nf, const WinSpan *__restrict__ wtab,
                                                                      const uint16_t *__restrict__ wcode,
                                                                      const LinkMap *__restrict__ maps,
                                                                      CollideParams p, int32_t *err) {
    using T = typename Store<ST>::T;
    using L = WinStage<Q, T>;
    static_assert(Q - 1 <= 32, "one lane per direction");
    extern __shared__ __align__(128) unsigned char wsm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(wsm + (size_t)NSTAGE * L::BYTES);
    uint64_t *empty = full + NSTAGE;
    volatile int32_t *stop = reinterpret_cast<volatile int32_t *>(empty + NSTAGE);
    const int tid = threadIdx.x;
    const int32_t n_tiles = S / WIN_TILE;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], WIN_TILE);
        }
        *stop = 0;
        mbar_init_fence();
    }
    __syncthreads();
    if (tid >= WIN_TILE) {
        // ------------------------------------------------------- producer warp
        const int lane = tid - WIN_TILE;
        uint32_t issued = 0;                         // lane 0: stages whose last copies may be in flight
        uint32_t parity = 0;                         // lane 0: parity of each stage's last issued phase
        auto table_of = [&](int32_t t) -> WinSpan {
            return (t < n_tiles && lane < Q - 1) ? wtab[(int64_t)t * (Q - 1) + lane] : WinSpan{0, 0, 0, 0};
        };
        WinSpan w = table_of(blockIdx.x);
        int j = 0;
        for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
            const int s = j % NSTAGE;
            const WinSpan wn = table_of(t + gridDim.x);   // the next tile's entry, in flight meanwhile
            if (j >= NSTAGE) {                       // the compute warps released stage s
                const bool ok = mbar_wait_or_stop(&empty[s], (uint32_t)((j / NSTAGE) - 1) & 1u, stop);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0 && !*stop) {
                        latch(err, ERR_STAGE_TIMEOUT);
                        *stop = 1;
                    }
                    break;
                }
                fence_proxy_async_smem();            // their reads of stage s before the copies overwrite it
            }
            unsigned char *st = wsm + (size_t)s * L::BYTES;
            const bool dir = lane < Q - 1;
            uint32_t bytes = 0;
            if (dir) bytes += WIN_TILE * 2 + WIN_TILE * sizeof(T) + (uint32_t)(w.len + w.len2) * sizeof(T);
            if (lane == 0) bytes += WIN_TILE * sizeof(T) + (Q - 1) * sizeof(WinSpan);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[s], bytes);
                issued |= 1u << s;
                parity = (parity & ~(1u << s)) | ((uint32_t)((j / NSTAGE) & 1) << s);
            }
            __syncwarp();
            if (dir) {
                const int r = lane;
                bulk_g2s(st + L::CODE + r * WIN_TILE * 2, wcode + (int64_t)r * S + (int64_t)t * WIN_TILE, WIN_TILE * 2,
                         &full[s]);
                bulk_g2s(st + L::POP + r * WIN_TILE * sizeof(T), pdf + (int64_t)r * S + (int64_t)t * WIN_TILE,
                         WIN_TILE * sizeof(T), &full[s]);
                if (w.len > 0)
                    bulk_g2s(st + L::POP + (L::OWN_ELEMS + r * WIN_CELLS) * sizeof(T),
                             pdf + (int64_t)inv(r + 1) * S + w.first, (uint32_t)w.len * sizeof(T), &full[s]);
                if (w.len2 > 0)
                    bulk_g2s(st + L::POP + (L::WIN2_ELEMS + r * WIN2_CELLS) * sizeof(T),
                             pdf + (int64_t)inv(r + 1) * S + w.first2, (uint32_t)w.len2 * sizeof(T), &full[s]);
            }
            if (lane == 0) {
                bulk_g2s(st + L::POP + (Q - 1) * WIN_TILE * sizeof(T),
                         pdf + (int64_t)(Q - 1) * S + (int64_t)t * WIN_TILE, WIN_TILE * sizeof(T), &full[s]);
                bulk_g2s(st + L::TAB, wtab + (int64_t)t * (Q - 1), (Q - 1) * sizeof(WinSpan), &full[s]);
            }
            w = wn;
        }
        // the copies of every issued stage land before the CTA may exit
        if (lane == 0) {
#pragma unroll
            for (int s = 0; s < NSTAGE; ++s)
                if (issued >> s & 1u) mbar_wait_bounded(&full[s], parity >> s & 1u);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- compute warps
        int j = 0;
        for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
            const int s = j % NSTAGE;
            const bool ok = mbar_wait_or_stop(&full[s], (uint32_t)(j / NSTAGE) & 1u, stop);
            if (!ok) {
                if (!*stop) {
                    latch(err, ERR_STAGE_TIMEOUT);
                    *stop = 1;
                }
                break;
            }
            const int32_t k = t * WIN_TILE + tid;
            if (k < nf) window_cell<Q, ST, HAS_BC>(pdf, R, wsm + (size_t)s * L::BYTES, tid, k, S, maps, p);
            mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
}

}  // namespace slbm
