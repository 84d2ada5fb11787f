// pool.cu -- batched stepping of many sparse domains (the method's AA update,
// Sec. 5.1, over the concatenation of the member domains' compacted cell
// lists).
//
// The pool keeps a device table of its members: PDF-list, odd-step slot
// list, link maps, stride, cell count, tile offset, the parity of the member
// at the start of the current launch sequence, and the member's collision
// constants.  The member owning a tile decides, by its parity, between the
// cell-local even update and the index-driven odd update, so members at
// different parities can share a launch.
//
// Two launch variants.  Tile grid (default): one CTA per tile of a group of
// members, the group's member table passed as a kernel parameter; members at
// or above a cell threshold run their own single-domain kernels in the same
// sequence; graphs of the groups are re-captured after membership changes.
// Persistent walker (ctas_per_sm > 0): the grid size and the table address
// never change, so a captured CUDA graph of K launches stays valid when
// members join or leave; the host rewrites the table (stream-ordered)
// instead.  A host-mapped abort word is polled every few tiles; a raised flag
// makes every CTA stop early and the next synchronising pool call reports
// SLBM_EABORTED.
#include <cstring>
#include <mutex>
#include <tuple>
#include <vector>

#include "aa_kernels.cuh"
#include "internal.h"

namespace slbm {

struct PoolEntry {
    void *pdf;
    const int32_t *R;
    const LinkMap *maps;
    int32_t S, nf, n_links, tile_begin, n_tiles, parity0;
    CollideParams p;
};

struct PoolHeader {
    int32_t n_dom, total_tiles;
};

template <int Q, int ST>
__device__ __forceinline__ void even_cell(typename Store<ST>::T *__restrict__ pdf, int32_t S, int32_t k,
                                          const CollideParams &p) {
    using St = Store<ST>;
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = St::raw(pdf[i * S + k]);
    collide<Q, St::scaled>(g, p);
#pragma unroll
    for (int i = 0; i < Q; ++i) pdf[inv(i) * S + k] = St::pack(g[i]);
}

// Each CTA takes one contiguous range of global tiles, so it changes member
// rarely: the member entry is found once by binary search and then followed
// forward, and copied into shared memory only when the member changes.  The
// host-mapped abort word is read every ABORT_POLL tiles.
constexpr int ABORT_POLL = 32;

// PARITY 0 / 1: every member is at that parity in this launch (the common
// case: members join at step 0 and are stepped in even chunks); -1: each
// member's own parity decides per tile.  UNI: every member has the same
// collision constants, passed as the kernel parameter `up` (read from the
// constant bank) instead of from the shared-memory copy of the entry.
template <int Q, int ST, int PARITY, bool UNI>
__global__ void __launch_bounds__(128, 4) pool_step_kernel(const PoolHeader *__restrict__ hdr,
                                                        const PoolEntry *__restrict__ tab, int32_t seq_step,
                                                        const volatile int32_t *abort_flag, int32_t *status,
                                                        const __grid_constant__ CollideParams up) {
    using T = typename Store<ST>::T;
    __shared__ PoolEntry sE;
    __shared__ int32_t s_dom, s_next, s_stop;
    const int32_t n_dom = hdr->n_dom, total = hdr->total_tiles;
    const int tile = blockDim.x;
    const int32_t per = (total + gridDim.x - 1) / gridDim.x;
    const int32_t t_lo = blockIdx.x * per, t_hi = min(total, t_lo + per);
    if (t_lo >= t_hi) return;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_dom - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab[mid].tile_begin <= t_lo) lo = mid;
            else hi = mid - 1;
        }
        s_dom = lo;
        s_next = lo + 1 < n_dom ? tab[lo + 1].tile_begin : total;
        s_stop = 0;
    }
    __syncthreads();
    constexpr int words = (int)(sizeof(PoolEntry) / 4);
    {   // cooperative copy of the first member entry
        const int32_t *src = reinterpret_cast<const int32_t *>(&tab[s_dom]);
        int32_t *dst = reinterpret_cast<int32_t *>(&sE);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
#pragma unroll 1
    for (int32_t t = t_lo; t < t_hi; ++t) {
        if (t >= s_next) {            // crossed into the next member (uniform)
            __syncthreads();
            if (threadIdx.x == 0) {
                int d = s_dom;
                while (d + 1 < n_dom && tab[d + 1].tile_begin <= t) ++d;
                s_dom = d;
                s_next = d + 1 < n_dom ? tab[d + 1].tile_begin : total;
            }
            __syncthreads();
            const int32_t *src = reinterpret_cast<const int32_t *>(&tab[s_dom]);
            int32_t *dst = reinterpret_cast<int32_t *>(&sE);
            for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
            __syncthreads();
        }
        if (((t - t_lo) % ABORT_POLL) == 0) {
            if (threadIdx.x == 0 && abort_flag && *abort_flag) {
                atomicCAS(status, 0, (int32_t)SLBM_EABORTED);
                s_stop = 1;
            }
            __syncthreads();
            if (s_stop) break;
        }
        const int32_t S = sE.S;
        const int32_t k = (t - sE.tile_begin) * tile + threadIdx.x;
        if (k < sE.nf) {
            T *pdf = reinterpret_cast<T *>(sE.pdf);
            const int parity = PARITY >= 0 ? PARITY : ((sE.parity0 + seq_step) & 1);
            if (parity == 0) {
                if constexpr (UNI) even_cell<Q, ST>(pdf, S, k, up);
                else even_cell<Q, ST>(pdf, S, k, sE.p);
            } else {
                const int32_t *R = sE.R;
                int32_t e[Q];
                e[0] = 0;
#pragma unroll
                for (int i = 1; i < Q; ++i) e[i] = __ldg(R + (i - 1) * S + k);
                // one link-aware path: members without inlet/outlet links
                // never take its branch
                if constexpr (UNI) odd_cell<Q, ST, true>(pdf, e, k, S, sE.maps, up);
                else odd_cell<Q, ST, true>(pdf, e, k, S, sE.maps, sE.p);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tile-grid variant (the default): one CTA per tile of the concatenated cell
// lists of a group of members.  Two tilings: 256-cell tiles for the
// cell-local even step (128 threads x 2 consecutive cells, vector accesses)
// and 128-cell tiles for the odd step and for launches that mix parities (128
// threads x 1 cell).  Every 256th CTA reads the host-mapped abort word and
// raises a device stop word; every CTA tests the stop word before its first
// store.
constexpr int POOL_THREADS = 128;

// The members of one launch (a group), passed by value as a kernel parameter
// (constant bank): member m owns the launch's tiles first_tile[m] ..
// first_tile[m+1]-1.  A CTA finds its member by a binary search over
// first_tile -- no dependent global load before its cells' loads.
constexpr int PT_MAX = 256;
struct PoolTable {
    int32_t n;                         // members
    int32_t first_tile[PT_MAX + 1];    // [n] = tiles of the launch
    void *pdf[PT_MAX];
    const int32_t *R[PT_MAX];
    int32_t S[PT_MAX], nf[PT_MAX], row[PT_MAX];   // row: the member's row in the pool table
};

__device__ __forceinline__ int pt_member(const PoolTable &T, int32_t t) {
    int lo = 0, hi = T.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.first_tile[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// PARITY: 0 / 1 uniform, -1 mixed (per member, from its table row).
// UNI: uniform collision constants in `up`.  BC: handle inlet/outlet links.
// CPT: cells per thread (2 only for the uniform even step, collided in pairs).
// pf_dist > 0 (odd step): thread 0 also asks the bulk-copy engine to
// prefetch into L2 the slot-list rows of the tile pf_dist ahead (about one
// residency wave later).
template <int Q, int ST, int PARITY, bool UNI, bool BC, int CPT>
__global__ void __launch_bounds__(POOL_THREADS) pool_tile_kernel(const PoolEntry *__restrict__ tab,
                                                                 const __grid_constant__ PoolTable pt,
                                                                 int32_t seq_step,
                                                                 const volatile int32_t *abort_flag,
                                                                 int32_t *stop,
                                                                 const __grid_constant__ CollideParams up,
                                                                 int32_t pf_dist) {
    using St = Store<ST>;
    using T = typename St::T;
    constexpr int32_t TILE = POOL_THREADS * CPT;
    const int32_t t = blockIdx.x;
    if (PARITY == 1 && pf_dist > 0 && threadIdx.x == 0 && t + pf_dist < pt.first_tile[pt.n]) {
        const int mf = pt_member(pt, t + pf_dist);
        const int32_t first = (t + pf_dist - pt.first_tile[mf]) * TILE;
        const int32_t left = pt.nf[mf] - first;
        if (left > 0) {
            const int32_t cells = ((left < TILE ? left : TILE) + 3) & ~3;   // whole 16 bytes
#pragma unroll
            for (int r = 0; r < Q - 1; ++r) bulk_prefetch_l2(pt.R[mf] + r * pt.S[mf] + first, (uint32_t)cells * 4u);
        }
    }
    // The stop word is tested only once the first loads of the tile are in
    // flight (a halted CTA still writes nothing), so its latency overlaps them.
    int32_t halt = *(volatile int32_t *)stop;
    if ((t & 255) == 0 && abort_flag && *abort_flag) {
        if (threadIdx.x == 0) atomicCAS(stop, 0, (int32_t)SLBM_EABORTED);
        halt = 1;
    }
    const int m = pt_member(pt, t);
    struct {
        int32_t first, member;
        const int32_t *R;
    } D{(t - pt.first_tile[m]) * TILE, pt.row[m], pt.R[m]};
    const CollideParams &p = UNI ? up : tab[D.member].p;
    T *pdf = reinterpret_cast<T *>(pt.pdf[m]);
    const int32_t S = pt.S[m], nf = pt.nf[m];
    int parity = PARITY;
    if (PARITY < 0) parity = (tab[D.member].parity0 + seq_step) & 1;
    if (parity == 0) {
        const int32_t k0 = D.first + CPT * threadIdx.x;
        if (k0 >= nf) return;
        float g[CPT][Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Vec<T, CPT> x = ldg_vec<T, CPT>(pdf + i * S + k0);   // own slots only: read-only path
#pragma unroll
            for (int c = 0; c < CPT; ++c) g[c][i] = St::raw(x.v[c]);
        }
        asm volatile("" ::: "memory");       // the loads above stay ahead of the test
        if (halt) return;
        collide_cells<Q, St::scaled, OP_TRT, CPT, CPT % 2 == 0>(g, p);   // pairs when CPT = 2
        const bool full = k0 + CPT <= nf;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Vec<T, CPT> y;
#pragma unroll
            for (int c = 0; c < CPT; ++c) y.v[c] = St::pack(g[c][i]);
            T *dst = pdf + inv(i) * S + k0;
            if (full) {
                st_vec<T, CPT>(dst, y);
            } else {
#pragma unroll
                for (int c = 0; c < CPT; ++c)
                    if (k0 + c < nf) dst[c] = y.v[c];
            }
        }
    } else {
        const int32_t k = D.first + threadIdx.x;
        if (k >= nf) return;
        int32_t e[Q];
        e[0] = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) e[i] = __ldg(D.R + (i - 1) * S + k);
        asm volatile("" ::: "memory");       // the loads above stay ahead of the test
        if (halt) return;
        // members without links never take the link branch of the BC path
        odd_cell<Q, ST, BC>(pdf, e, k, S, BC ? tab[D.member].maps : nullptr, p);
    }
}

using TileKernel = void (*)(const PoolEntry *, const PoolTable, int32_t, const volatile int32_t *, int32_t *,
                            const CollideParams, int32_t);

// mode: 0 mixed parity, 1 + 2*parity + uni
template <int Q, int ST>
static TileKernel tile_kernel_st(int mode, bool bc) {
    switch (mode) {
        case 1: return pool_tile_kernel<Q, ST, 0, false, false, 2>;
        case 2: return pool_tile_kernel<Q, ST, 0, true, false, 2>;
        case 3: return bc ? pool_tile_kernel<Q, ST, 1, false, true, 1> : pool_tile_kernel<Q, ST, 1, false, false, 1>;
        case 4: return bc ? pool_tile_kernel<Q, ST, 1, true, true, 1> : pool_tile_kernel<Q, ST, 1, true, false, 1>;
        default: return pool_tile_kernel<Q, ST, -1, false, true, 1>;
    }
}

template <int Q>
static TileKernel tile_kernel_for(int storage, int mode, bool bc) {
    switch (storage) {
        case SLBM_FP32: return tile_kernel_st<Q, ST_F32>(mode, bc);
        case SLBM_FP16: return tile_kernel_st<Q, ST_F16>(mode, bc);
        default: return tile_kernel_st<Q, ST_BF16>(mode, bc);
    }
}

using PoolKernel = void (*)(const PoolHeader *, const PoolEntry *, int32_t, const volatile int32_t *, int32_t *,
                            const CollideParams);

// mode: 0 generic, 1 + 2*parity + uni (parity-uniform variants)
template <int Q, int ST>
static PoolKernel pool_kernel_st(int mode) {
    switch (mode) {
        case 1: return pool_step_kernel<Q, ST, 0, false>;
        case 2: return pool_step_kernel<Q, ST, 0, true>;
        case 3: return pool_step_kernel<Q, ST, 1, false>;
        case 4: return pool_step_kernel<Q, ST, 1, true>;
        default: return pool_step_kernel<Q, ST, -1, false>;
    }
}

template <int Q>
static PoolKernel pool_kernel_for(int storage, int mode) {
    switch (storage) {
        case SLBM_FP32: return pool_kernel_st<Q, ST_F32>(mode);
        case SLBM_FP16: return pool_kernel_st<Q, ST_F16>(mode);
        default: return pool_kernel_st<Q, ST_BF16>(mode);
    }
}

}  // namespace slbm

using namespace slbm;

struct slbm_pool {
    int32_t q = 19, storage = SLBM_FP32, capacity = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<slbm_t *> members;       // by slot; nullptr = free
    std::vector<PoolEntry> host_tab;     // staged table (active members, sorted)
    std::vector<int32_t> order;          // slot of each table row
    PoolHeader host_hdr{0, 0};
    void *d_tab = nullptr, *d_hdr = nullptr, *d_status = nullptr, *d_red = nullptr;
    std::vector<PoolTable> ptab;                 // per group: [2g] 256-cell, [2g+1] 128-cell tiling
    int32_t *h_abort = nullptr;          // host-mapped abort word
    int32_t *d_abort = nullptr;
    bool dirty = true;
    bool table_ok = false;               // the device table and tiles match host_tab
    // extra streams of a graph step: the batched groups and the large members
    // are spread over the pool's stream and these, forked from and joined
    // back into the pool's stream, so one member's tail overlaps another's
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_join;
    cudaEvent_t fork = nullptr;
    int32_t threads = 64, ctas_per_sm = 0;   // ctas_per_sm > 0: persistent walker
    unsigned grid[5] = {0, 0, 0, 0, 0};      // persistent grid of each kernel variant
    int32_t pf_dist = 0;                 // odd tile kernel: L2 prefetch distance (resident CTAs)
    int64_t split = 1 << 19;             // members with >= split cells step with their own kernels
    std::vector<int32_t> big;            // slots of those members
    // L2 groups: consecutive table rows whose summed state + index bytes stay
    // within group_bytes; a group takes all k steps of a pool step before the
    // next one starts, so a group that fits in L2 streams from L2 (0: one
    // group of all rows)
    int64_t group_bytes = 48ll << 20;
    struct Group { int32_t r0, r1, t0[2], nt[2]; };
    std::vector<Group> groups;
    int32_t p0 = -1;                     // common parity of all members, or -1
    bool uni = false;                    // all members share collision constants
    bool any_links = false;              // some member has inlet/outlet links
    CollideParams up{};                  // those constants
    // (k, p0, uni) -> exec; the uniform constants a graph was captured with
    std::map<std::tuple<int, int, int>, std::pair<cudaGraphExec_t, CollideParams>> graphs;
};

namespace {

slbm_status perr(slbm_status s, const std::string &m) {
    set_error(s, m);
    return s;
}

slbm_status pcuda(cudaError_t e, const char *what) {
    cudaGetLastError();
    return perr(SLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void drop_pool_graphs(slbm_pool *p) {
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second.first);
    p->graphs.clear();
}

PoolKernel kernel_of(const slbm_pool *p, int mode) {
    return p->q == 19 ? pool_kernel_for<19>(p->storage, mode) : pool_kernel_for<27>(p->storage, mode);
}

// Persistent grid of each variant: SMs x its resident CTAs (capped by
// ctas_per_sm).  It depends on the variant only, never on the membership.
slbm_status size_grid(slbm_pool *p) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int mode = 0; mode <= 4; ++mode) {
        int c = 1;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kernel_of(p, mode), p->threads, 0);
        if (e != cudaSuccess) return pcuda(e, "occupancy");
        c = std::max(c, 1);
        if (p->ctas_per_sm > 0) c = std::min(c, p->ctas_per_sm);
        p->grid[mode] = (unsigned)(std::max(sms, 1) * c);
    }
    int c = 1;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &c, p->q == 19 ? tile_kernel_for<19>(p->storage, 4, false) : tile_kernel_for<27>(p->storage, 4, false),
        POOL_THREADS, 0);
    if (e != cudaSuccess) return pcuda(e, "occupancy");
    p->pf_dist = std::max(sms, 1) * std::max(c, 1);
    return SLBM_OK;
}

// Rebuild and upload the table (stream-ordered) when membership or parities
// changed.
slbm_status sync_table(slbm_pool *p) {
    for (size_t r = 0; r < p->order.size() && !p->dirty; ++r)   // a member stepped outside the pool
        if (p->members[p->order[r]] && (int32_t)(p->members[p->order[r]]->d.step & 1) != p->host_tab[r].parity0)
            p->dirty = true;
    if (!p->dirty) return SLBM_OK;
    std::vector<PoolEntry> prev_tab;
    std::vector<int32_t> prev_order;
    prev_tab.swap(p->host_tab);
    prev_order.swap(p->order);
    p->big.clear();
    int32_t tile = 0;
    for (int32_t s = 0; s < p->capacity; ++s) {
        slbm_t *h = p->members[s];
        if (!h) continue;
        const Domain &d = h->d;
        if (p->ctas_per_sm == 0 && p->split > 0 && d.n_fluid >= p->split) {
            p->big.push_back(s);
            continue;
        }
        PoolEntry E{};
        E.pdf = d.pdf.p;
        E.R = (const int32_t *)d.P.p;
        E.maps = (const LinkMap *)d.link_map.p;
        E.S = (int32_t)d.S;
        E.nf = (int32_t)d.n_fluid;
        E.n_links = (int32_t)d.n_links;
        const int32_t tcells = p->ctas_per_sm > 0 ? p->threads : POOL_THREADS;
        E.n_tiles = (int32_t)((d.n_fluid + tcells - 1) / tcells);
        E.tile_begin = tile;
        E.parity0 = (int32_t)(d.step & 1);
        E.p = d.collide_params();
        if (E.n_tiles == 0) continue;
        tile += E.n_tiles;
        p->host_tab.push_back(E);
        p->order.push_back(s);
    }
    p->host_hdr = PoolHeader{(int32_t)p->host_tab.size(), tile};
    p->p0 = p->host_tab.empty() ? 0 : p->host_tab[0].parity0;
    p->uni = !p->host_tab.empty();
    p->any_links = false;
    for (const PoolEntry &E : p->host_tab) {
        if (E.n_links > 0) p->any_links = true;
        if (E.parity0 != p->p0) p->p0 = -1;
        if (std::memcmp(&E.p, &p->host_tab[0].p, sizeof(CollideParams)) != 0) p->uni = false;
    }
    p->up = p->host_tab.empty() ? CollideParams{} : p->host_tab[0].p;
    // first tile of every row in both tilings, and the L2 groups over them
    const int32_t cells[2] = {2 * POOL_THREADS, POOL_THREADS};
    const size_t nrow = p->host_tab.size();
    std::vector<int32_t> begin[2] = {std::vector<int32_t>(nrow + 1), std::vector<int32_t>(nrow + 1)};
    for (int v = 0; v < 2; ++v) {
        int32_t n = 0;
        for (size_t r = 0; r < nrow; ++r) {
            begin[v][r] = n;
            n += (p->host_tab[r].nf + cells[v] - 1) / cells[v];
        }
        begin[v][nrow] = n;
    }
    p->groups.clear();
    {
        const int64_t elt = p->storage == SLBM_FP32 ? 4 : 2;
        int64_t acc = 0;
        for (size_t r = 0; r < nrow; ++r) {
            const PoolEntry &E = p->host_tab[r];
            const int64_t bytes = (int64_t)E.S * (p->q * elt + (p->q - 1) * 4) + (int64_t)E.n_links * sizeof(LinkMap);
            if (p->groups.empty() || (p->group_bytes > 0 && acc + bytes > p->group_bytes) ||
                (int32_t)r - p->groups.back().r0 >= PT_MAX) {
                p->groups.push_back({(int32_t)r, (int32_t)r, {begin[0][r], begin[1][r]}, {0, 0}});
                acc = 0;
            }
            acc += bytes;
            slbm_pool::Group &G = p->groups.back();
            G.r1 = (int32_t)r + 1;
            for (int v = 0; v < 2; ++v) G.nt[v] = begin[v][r + 1] - G.t0[v];
        }
    }
    // each group's member table, for both tilings (kernel parameters)
    p->ptab.assign(2 * p->groups.size(), PoolTable{});
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        const slbm_pool::Group &G = p->groups[gi];
        for (int v = 0; v < 2; ++v) {
            PoolTable &T = p->ptab[2 * gi + v];
            T.n = G.r1 - G.r0;
            for (int32_t r = G.r0; r < G.r1; ++r) {
                const PoolEntry &E = p->host_tab[r];
                const int j = r - G.r0;
                T.first_tile[j] = begin[v][r] - G.t0[v];
                T.pdf[j] = E.pdf;
                T.R[j] = E.R;
                T.S[j] = E.S;
                T.nf[j] = E.nf;
                T.row[j] = r;
            }
            T.first_tile[T.n] = G.nt[v];
        }
    }
    // the batched table is unchanged (only large members came or went): the
    // device table, the tiles and the batched graphs stay valid
    static_assert(sizeof(PoolEntry) == 48 + sizeof(CollideParams), "PoolEntry has no padding");
    if (p->table_ok && prev_order == p->order && prev_tab.size() == p->host_tab.size() &&
        (prev_tab.empty() || std::memcmp(prev_tab.data(), p->host_tab.data(), prev_tab.size() * sizeof(PoolEntry)) == 0)) {
        p->dirty = false;
        return SLBM_OK;
    }
    p->table_ok = false;
    cudaError_t e = cudaSuccess;
    if (!p->host_tab.empty())
        e = cudaMemcpyAsync(p->d_tab, p->host_tab.data(), p->host_tab.size() * sizeof(PoolEntry),
                            cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_hdr, &p->host_hdr, sizeof(PoolHeader), cudaMemcpyHostToDevice, p->stream);
    // pageable source: make sure the copy has consumed the staging arrays
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return pcuda(e, "pool table upload");
    if (p->ctas_per_sm == 0) drop_pool_graphs(p);   // the tile grid follows the membership
    p->dirty = false;
    p->table_ok = true;
    return SLBM_OK;
}

cudaError_t launch_one(slbm_pool *p, int32_t t, const slbm_pool::Group *g);

// Boundary fix-ups (before: post = 0, after: post = 1) of the members of rows
// [r0, r1) that take an even step in launch t and have inlet/outlet links.
cudaError_t member_fixups(slbm_pool *p, int32_t t, int post, int32_t r0, int32_t r1) {
    if (!p->any_links) return cudaSuccess;
    for (int32_t r = r0; r < r1; ++r) {
        const PoolEntry &E = p->host_tab[r];
        if (E.n_links == 0 || ((E.parity0 + t) & 1) != 0) continue;
        const cudaError_t e = launch_bc_fixup(p->members[p->order[r]]->d, post, p->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// k steps of every L2 group of batched members, group after group.
cudaError_t launch_groups(slbm_pool *p, int32_t k) {
    for (const slbm_pool::Group &g : p->groups) {
        for (int32_t t = 0; t < k; ++t) {
            cudaError_t e = member_fixups(p, t, 0, g.r0, g.r1);
            if (e == cudaSuccess) e = launch_one(p, t, &g);
            if (e == cudaSuccess) e = member_fixups(p, t, 1, g.r0, g.r1);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// k steps of every large member with its own kernels, member after member:
// launched directly, or as each member's own cached graph (which outlives
// changes of the pool's membership).
cudaError_t launch_big(slbm_pool *p, int32_t k, bool graph) {
    // with extra streams: each member on the stream with the fewest cells so
    // far (the batched groups count on the pool's stream)
    std::vector<int64_t> load(p->aux.size() + 1, 0);
    if (graph)
        for (const PoolEntry &E : p->host_tab) load[0] += E.nf;
    for (int32_t s : p->big) {
        Domain &d = p->members[s]->d;
        if (graph) {
            size_t j = 0;
            for (size_t c = 1; c < load.size(); ++c)
                if (load[c] < load[j]) j = c;
            load[j] += d.n_fluid;
            cudaGraphExec_t ex = nullptr;
            cudaError_t e = domain_graph(d, k, &ex);
            if (e == cudaSuccess) e = cudaGraphLaunch(ex, j == 0 ? p->stream : p->aux[j - 1]);
            if (e != cudaSuccess) return e;
            continue;
        }
        for (int32_t t = 0; t < k; ++t) {
            const cudaError_t e = launch_aa_step(d, (int)((d.step + t) & 1), p->stream);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Every extra stream waits for the work queued so far on the pool's stream.
cudaError_t fork_aux(slbm_pool *p) {
    cudaError_t e = cudaEventRecord(p->fork, p->stream);
    for (size_t j = 0; j < p->aux.size() && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(p->aux[j], p->fork, 0);
    return e;
}

// The pool's stream waits for the work on every extra stream.
cudaError_t join_aux(slbm_pool *p) {
    for (size_t j = 0; j < p->aux.size(); ++j) {
        cudaError_t e = cudaEventRecord(p->aux_join[j], p->aux[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->aux_join[j], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void free_aux(slbm_pool *p) {
    for (cudaStream_t a : p->aux) cudaStreamDestroy(a);
    for (cudaEvent_t ev : p->aux_join) cudaEventDestroy(ev);
    p->aux.clear();
    p->aux_join.clear();
}

// Launches of k steps, group-major: each L2 group of small members takes its
// k batched steps (with the boundary fix-ups of its members at an even step),
// then every large member its k own AA steps (which bring their own
// fix-ups).  Launch t of a member is its step (step at sequence start + t);
// members are independent, so the order across members changes no result.
cudaError_t launch_seq(slbm_pool *p, int32_t k) {
    if (p->ctas_per_sm > 0) {            // persistent walker: the whole table per launch
        for (int32_t t = 0; t < k && !p->host_tab.empty(); ++t) {
            cudaError_t e = member_fixups(p, t, 0, 0, (int32_t)p->host_tab.size());
            if (e == cudaSuccess) e = launch_one(p, t, nullptr);
            if (e == cudaSuccess) e = member_fixups(p, t, 1, 0, (int32_t)p->host_tab.size());
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const cudaError_t e = launch_groups(p, k);
    return e != cudaSuccess ? e : launch_big(p, k, false);
}

cudaError_t launch_one(slbm_pool *p, int32_t t, const slbm_pool::Group *g) {
    const int mode = p->p0 < 0 ? 0 : 1 + 2 * ((p->p0 + t) & 1) + (p->uni ? 1 : 0);
    if (p->ctas_per_sm == 0) {
        TileKernel tk = p->q == 19 ? tile_kernel_for<19>(p->storage, mode, p->any_links)
                                   : tile_kernel_for<27>(p->storage, mode, p->any_links);
        const int v = (mode == 1 || mode == 2) ? 0 : 1;      // uniform even step: 256-cell tiles
        const int32_t nt = g->nt[v];
        if (nt == 0) return cudaSuccess;
        const int32_t pf = (mode == 3 || mode == 4) ? p->pf_dist : 0;
        const size_t gi = (size_t)(g - p->groups.data());
        tk<<<(unsigned)nt, POOL_THREADS, 0, p->stream>>>((const PoolEntry *)p->d_tab, p->ptab[2 * gi + v], t,
                                                          p->d_abort, (int32_t *)p->d_status, p->up, pf);
        return cudaGetLastError();
    }
    PoolKernel kern = kernel_of(p, mode);
    kern<<<p->grid[mode], p->threads, 0, p->stream>>>((const PoolHeader *)p->d_hdr, (const PoolEntry *)p->d_tab, t,
                                                p->d_abort, (int32_t *)p->d_status, p->up);
    return cudaGetLastError();
}

}  // namespace

namespace slbm {

void pool_forget_member(::slbm_pool *p, ::slbm_domain *h) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);   // queued pool work on the member ends first
    for (auto &m : p->members)
        if (m == h) {
            m = nullptr;
            p->dirty = true;
        }
}

}  // namespace slbm

extern "C" {

slbm_status slbm_pool_create(int32_t q, int32_t storage, int32_t capacity, void *stream, slbm_pool_t **out) {
    if (!out) return perr(SLBM_EINVAL, "out must be non-NULL");
    *out = nullptr;
    if (q != 19 && q != 27) return perr(SLBM_EINVAL, "q must be 19 or 27");
    if (storage < SLBM_FP32 || storage > SLBM_BF16) return perr(SLBM_EINVAL, "bad storage");
    if (capacity < 1 || capacity > 65536) return perr(SLBM_EINVAL, "capacity must be 1..65536");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return perr(SLBM_ECUDA, "no CUDA device available (there is no CPU fallback)");
    }
    slbm_pool *p = new slbm_pool();
    p->q = q;
    p->storage = storage;
    p->capacity = capacity;
    p->members.assign(capacity, nullptr);
    cudaError_t e = cudaSuccess;
    if (stream) {
        p->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreate(&p->stream);
        p->own_stream = true;
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tab, (size_t)capacity * sizeof(PoolEntry));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_hdr, sizeof(PoolHeader));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_red, (size_t)capacity * 7 * sizeof(double));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&p->h_abort, sizeof(int32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *p->h_abort = 0;
        e = cudaHostGetDevicePointer((void **)&p->d_abort, p->h_abort, 0);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_hdr, 0, sizeof(PoolHeader), p->stream);
    slbm_status st = e == cudaSuccess ? size_grid(p) : pcuda(e, "pool create");
    if (st == SLBM_OK) {
        e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) st = pcuda(e, "pool create sync");
    }
    if (st != SLBM_OK) {
        const std::string m = sparse_lbm_last_error();
        slbm_pool_free(p);
        return perr(st, m);
    }
    *out = p;
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_add(slbm_pool_t *p, slbm_t *h, int32_t *slot) {
    if (!p || !h || !slot) return perr(SLBM_EINVAL, "null argument");
    const Domain &d = h->d;
    if (d.layout != SLBM_LAYOUT_SPARSE) return perr(SLBM_EUNSUPPORTED, "pool members must use the sparse layout");
    if (d.op != SLBM_SRT && d.op != SLBM_TRT) return perr(SLBM_EUNSUPPORTED, "pools step SRT/TRT members");
    if (d.q != p->q || d.storage != p->storage) return perr(SLBM_EINVAL, "member q / storage differ from the pool's");
    for (int32_t s = 0; s < p->capacity; ++s)
        if (p->members[s] == h) return perr(SLBM_EINVAL, "domain is already a member");
    for (int32_t s = 0; s < p->capacity; ++s) {
        if (!p->members[s]) {
            // order the domain's own stream before the pool's
            cudaStreamSynchronize(d.stream);
            p->members[s] = h;
            h->d.pools.push_back(p);
            p->dirty = true;
            *slot = s;
            set_error(SLBM_OK, "");
            return SLBM_OK;
        }
    }
    return perr(SLBM_ENOMEM, "pool is full");
}

slbm_status slbm_pool_remove(slbm_pool_t *p, int32_t slot) {
    if (!p || slot < 0 || slot >= p->capacity || !p->members[slot]) return perr(SLBM_EINVAL, "bad slot");
    const cudaError_t e = cudaStreamSynchronize(p->stream);   // member work done before it leaves
    std::vector<slbm_pool *> &ps = p->members[slot]->d.pools;
    auto it = std::find(ps.begin(), ps.end(), p);
    if (it != ps.end()) ps.erase(it);
    p->members[slot] = nullptr;
    p->dirty = true;
    if (e != cudaSuccess) return pcuda(e, "pool remove");
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_step(slbm_pool_t *p, int32_t k, int32_t use_graph) {
    const Range range_("slbm pool step");
    if (!p || k < 0) return perr(SLBM_EINVAL, "need a pool and k >= 0");
    if (k == 0) {
        set_error(SLBM_OK, "");
        return SLBM_OK;
    }
    slbm_status st = sync_table(p);
    if (st != SLBM_OK) return st;
    if (p->host_hdr.total_tiles > 0 || !p->big.empty()) {
        cudaError_t e = cudaSuccess;
        if (use_graph && p->ctas_per_sm == 0) {
            // the batched groups as the pool's graph, each large member as its own
            if (!p->aux.empty()) {
                e = fork_aux(p);
                if (e != cudaSuccess) return pcuda(e, "pool fork");
            }
            if (!p->host_tab.empty()) {
                const auto key = std::make_tuple((int)k, (int)p->p0, (p->uni ? 1 : 0) + (p->any_links ? 2 : 0));
                auto it = p->graphs.find(key);
                if (it != p->graphs.end() && p->uni &&
                    std::memcmp(&it->second.second, &p->up, sizeof(CollideParams)) != 0) {
                    cudaGraphExecDestroy(it->second.first);
                    p->graphs.erase(it);
                    it = p->graphs.end();
                }
                if (it == p->graphs.end()) {
                    cudaGraph_t g = nullptr;
                    e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
                    if (e != cudaSuccess) return pcuda(e, "begin capture");
                    const cudaError_t le = launch_groups(p, k);
                    e = cudaStreamEndCapture(p->stream, &g);
                    if (le != cudaSuccess) {
                        if (g) cudaGraphDestroy(g);
                        return pcuda(le, "pool launch during capture");
                    }
                    if (e != cudaSuccess) return pcuda(e, "end capture");
                    cudaGraphExec_t ex = nullptr;
                    e = cudaGraphInstantiate(&ex, g, 0);
                    cudaGraphDestroy(g);
                    if (e != cudaSuccess) return pcuda(e, "graph instantiate");
                    it = p->graphs.emplace(key, std::make_pair(ex, p->up)).first;
                }
                e = cudaGraphLaunch(it->second.first, p->stream);
            }
            if (e == cudaSuccess) e = launch_big(p, k, true);
            if (e == cudaSuccess && !p->aux.empty()) e = join_aux(p);
        } else if (use_graph) {
            const auto key = std::make_tuple((int)k, (int)p->p0, (p->uni ? 1 : 0) + (p->any_links ? 2 : 0));
            auto it = p->graphs.find(key);
            if (it != p->graphs.end() && p->uni &&
                std::memcmp(&it->second.second, &p->up, sizeof(CollideParams)) != 0) {
                cudaGraphExecDestroy(it->second.first);     // captured with other constants
                p->graphs.erase(it);
                it = p->graphs.end();
            }
            if (it == p->graphs.end()) {
                cudaGraph_t g = nullptr;
                e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) return pcuda(e, "begin capture");
                const cudaError_t le = launch_seq(p, k);
                e = cudaStreamEndCapture(p->stream, &g);
                if (le != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return pcuda(le, "pool launch during capture");
                }
                if (e != cudaSuccess) return pcuda(e, "end capture");
                cudaGraphExec_t ex = nullptr;
                e = cudaGraphInstantiate(&ex, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return pcuda(e, "graph instantiate");
                it = p->graphs.emplace(key, std::make_pair(ex, p->up)).first;
            }
            e = cudaGraphLaunch(it->second.first, p->stream);
        } else {
            e = launch_seq(p, k);
        }
        if (e != cudaSuccess) return pcuda(e, "pool step");
    }
    for (int32_t s = 0; s < p->capacity; ++s)
        if (p->members[s] && p->members[s]->d.n_fluid > 0) p->members[s]->d.step += k;
    if (k & 1) p->dirty = true;   // parities flipped
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_reduce(slbm_pool_t *p, double *out, int32_t mem) {
    const Range range_("slbm pool reduce");
    if (!p || !out) return perr(SLBM_EINVAL, "null argument");
    if (mem != SLBM_MEM_DEVICE && mem != SLBM_MEM_HOST) return perr(SLBM_EINVAL, "bad mem");
    cudaError_t e = cudaSuccess;
    double *dev_out = mem == SLBM_MEM_HOST ? (double *)p->d_red : out;
    const size_t bytes = (size_t)p->capacity * 5 * sizeof(double);
    e = cudaMemsetAsync(dev_out, 0, bytes, p->stream);
    for (int32_t s = 0; s < p->capacity && e == cudaSuccess; ++s) {
        slbm_t *h = p->members[s];
        if (h) e = launch_reduce(h->d, dev_out + 5 * s, p->stream);
    }
    int32_t status = 0;
    if (e == cudaSuccess && mem == SLBM_MEM_HOST) {
        e = cudaMemcpyAsync(out, dev_out, bytes, cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, p->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    }
    if (e != cudaSuccess) return pcuda(e, "pool reduce");
    if (status == SLBM_EABORTED) return perr(SLBM_EABORTED, "a pool launch was aborted by the host flag");
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_reduce_ext(slbm_pool_t *p, double *out, int32_t mem) {
    const Range range_("slbm pool reduce ext");
    if (!p || !out) return perr(SLBM_EINVAL, "null argument");
    if (mem != SLBM_MEM_DEVICE && mem != SLBM_MEM_HOST) return perr(SLBM_EINVAL, "bad mem");
    cudaError_t e = cudaSuccess;
    double *dev_out = mem == SLBM_MEM_HOST ? (double *)p->d_red : out;
    const size_t bytes = (size_t)p->capacity * 7 * sizeof(double);
    e = cudaMemsetAsync(dev_out, 0, bytes, p->stream);
    for (int32_t s = 0; s < p->capacity && e == cudaSuccess; ++s) {
        slbm_t *h = p->members[s];
        if (h) e = launch_reduce_ext(h->d, dev_out + 7 * s, p->stream);
    }
    int32_t status = 0;
    if (e == cudaSuccess && mem == SLBM_MEM_HOST) {
        e = cudaMemcpyAsync(out, dev_out, bytes, cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, p->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    }
    if (e != cudaSuccess) return pcuda(e, "pool reduce ext");
    if (status == SLBM_EABORTED) return perr(SLBM_EABORTED, "a pool launch was aborted by the host flag");
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_set_launch(slbm_pool_t *p, int32_t threads, int32_t ctas_per_sm) {
    if (!p) return perr(SLBM_EINVAL, "null pool");
    if (threads < 32 || threads > 128 || threads % 32) return perr(SLBM_EINVAL, "threads must be 32..128, multiple of 32");
    if (ctas_per_sm < 0) return perr(SLBM_EINVAL, "ctas_per_sm must be >= 0");
    p->threads = threads;
    p->ctas_per_sm = ctas_per_sm;
    p->dirty = true;
    p->table_ok = false;
    drop_pool_graphs(p);
    return size_grid(p);
}

slbm_status slbm_pool_set_split(slbm_pool_t *p, int64_t split_cells) {
    if (!p || split_cells < 0) return perr(SLBM_EINVAL, "need a pool and split_cells >= 0");
    const cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return pcuda(e, "pool split");
    p->split = split_cells;
    p->dirty = true;
    p->table_ok = false;
    drop_pool_graphs(p);
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_set_group_bytes(slbm_pool_t *p, int64_t bytes) {
    if (!p || bytes < 0) return perr(SLBM_EINVAL, "need a pool and bytes >= 0");
    const cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return pcuda(e, "pool group bytes");
    p->group_bytes = bytes;
    p->dirty = true;
    p->table_ok = false;
    drop_pool_graphs(p);
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_set_streams(slbm_pool_t *p, int32_t n) {
    if (!p || n < 1 || n > 16) return perr(SLBM_EINVAL, "need a pool and 1 <= n <= 16");
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return pcuda(e, "pool streams");
    free_aux(p);
    if (!p->fork) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    for (int32_t j = 1; j < n && e == cudaSuccess; ++j) {
        cudaStream_t a = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
        p->aux.push_back(a);
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) break;
        p->aux_join.push_back(ev);
    }
    if (e != cudaSuccess || p->aux.size() != p->aux_join.size()) {
        free_aux(p);
        return pcuda(e != cudaSuccess ? e : cudaErrorUnknown, "pool streams");
    }
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

slbm_status slbm_pool_abort(slbm_pool_t *p, int32_t raise) {
    if (!p) return perr(SLBM_EINVAL, "null pool");
    if (raise) {
        *(volatile int32_t *)p->h_abort = 1;
    } else {
        const cudaError_t e = cudaStreamSynchronize(p->stream);
        *(volatile int32_t *)p->h_abort = 0;
        if (e == cudaSuccess) {
            const cudaError_t e2 = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), p->stream);
            if (e2 != cudaSuccess) return pcuda(e2, "pool abort clear");
        } else {
            return pcuda(e, "pool abort clear");
        }
    }
    set_error(SLBM_OK, "");
    return SLBM_OK;
}

void slbm_pool_free(slbm_pool_t *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    for (cudaStream_t a : p->aux) cudaStreamSynchronize(a);
    free_aux(p);
    if (p->fork) cudaEventDestroy(p->fork);
    drop_pool_graphs(p);
    for (slbm_t *h : p->members) {          // the members stay valid; they leave the pool
        if (!h) continue;
        std::vector<slbm_pool *> &ps = h->d.pools;
        auto it = std::find(ps.begin(), ps.end(), p);
        if (it != ps.end()) ps.erase(it);
    }
    if (p->d_tab) cudaFree(p->d_tab);
    if (p->d_hdr) cudaFree(p->d_hdr);
    if (p->d_status) cudaFree(p->d_status);
    if (p->d_red) cudaFree(p->d_red);

    if (p->h_abort) cudaFreeHost(p->h_abort);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    cudaGetLastError();
    delete p;
}

}  // extern "C"
