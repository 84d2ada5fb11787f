/*
 * sparse_lbm.h -- C ABI of the GB300 sparse (indirect-addressing) lattice
 * Boltzmann library.
 *
 * The library implements the sparse data structure of Suffa et al., "Architecture
 * Specific Generation of Large Scale Lattice Boltzmann Methods for Sparse Complex
 * Geometries" (Sec. 3.1): only fluid cells are stored, in a compacted
 * direction-major PDF-list of Q rows, plus a pull index-list of Q-1 rows that
 * replaces the lost neighbourhood information, with no-slip and periodic
 * boundaries folded into the list (Sec. 3.1.1).  Time stepping uses the in-place
 * AA pattern (Sec. 5.1): a cell-local "even" step and an index-driven "odd" step
 * on one PDF field.  The collision is SRT (Eq. 5), TRT or D3Q19 MRT with the
 * second-order equilibrium (Eq. 6) and a Guo body force.  For the paper's
 * comparisons the same lists also drive a two-field pull layout (Sec. 5.1),
 * and a dense direct-addressing layout serves as the comparator (Sec. 4).
 * Populations are stored shifted (f_i - w_i) in FP32, FP16 or BF16; cells are
 * numbered lexicographically or in 8^3 bricks.  Pools step many domains
 * together (batching), for the serving layer above this ABI.
 *
 * Conventions shared by every call
 *   - Every call returns an slbm_status; nothing aborts or throws across the ABI.
 *     On failure, sparse_lbm_last_error() returns a thread-local message.
 *   - Device work is enqueued on the stream given at creation (a cudaStream_t
 *     passed as void*; NULL makes the library create a blocking stream of its
 *     own, which orders with the legacy default stream).  Calls that return
 *     host data synchronise that stream.
 *   - Device memory is owned by the library (optionally obtained through the
 *     caller's slbm_allocator).  Output buffers are owned by the caller.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns SLBM_ECUDA.
 *   - Voxel ids are x + nx*(y + ny*z) (x fastest).  Flag values: 0 fluid,
 *     1 no-slip wall, 2 velocity inlet, 3 pressure outlet.  A neighbour outside
 *     the box along a non-periodic axis counts as a wall.
 *   - Velocity-set order (part of the ABI; the index-list depends on it):
 *       0:(0,0,0)  1:(1,0,0)  2:(-1,0,0)  3:(0,1,0)  4:(0,-1,0)  5:(0,0,1)
 *       6:(0,0,-1) 7:(1,1,0)  8:(-1,-1,0) 9:(1,-1,0) 10:(-1,1,0) 11:(1,0,1)
 *       12:(-1,0,-1) 13:(1,0,-1) 14:(-1,0,1) 15:(0,1,1) 16:(0,-1,-1)
 *       17:(0,1,-1) 18:(0,-1,1), and for D3Q27 additionally 19:(1,1,1)
 *       20:(-1,-1,-1) 21:(1,1,-1) 22:(-1,-1,1) 23:(1,-1,1) 24:(-1,1,-1)
 *       25:(-1,1,1) 26:(1,-1,-1).  inverse(i) = i+1 for odd i, i-1 for even i>0.
 */
#ifndef SPARSE_LBM_H
#define SPARSE_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slbm_domain slbm_t;     /* opaque domain handle */
typedef struct slbm_pool slbm_pool_t;  /* opaque batch of domains */

typedef enum {
    SLBM_OK = 0,
    SLBM_EINVAL = 1,        /* invalid argument (dims, omega, q, pointer, size) */
    SLBM_ENOMEM = 2,        /* device allocation failed or budget exceeded */
    SLBM_ECUDA = 3,         /* a CUDA runtime call failed / no device */
    SLBM_EUNSUPPORTED = 4,  /* valid but not supported (e.g. Q*stride >= 2^31) */
    SLBM_EDIVERGED = 5,     /* a reduction produced NaN/Inf or |u| > 0.3 */
    SLBM_ETIMEOUT = 6,      /* a bounded device wait gave up */
    SLBM_EABORTED = 7,      /* the host abort flag was raised */
    SLBM_EDEVICE = 8        /* a device-side check latched an error (checked kernels) */
} slbm_status;

enum { SLBM_SRT = 0, SLBM_TRT = 1, SLBM_MRT = 2, SLBM_CM = 3, SLBM_CUMULANT = 4 };
enum { SLBM_FP32 = 0, SLBM_FP16 = 1, SLBM_BF16 = 2 };
enum { SLBM_LAYOUT_SPARSE = 0, SLBM_LAYOUT_DENSE = 1, SLBM_LAYOUT_SPARSE_PULL = 2 };
enum { SLBM_MEM_DEVICE = 0, SLBM_MEM_HOST = 1 };
enum { SLBM_ORDER_LEX = 0, SLBM_ORDER_BRICK8 = 1, SLBM_ORDER_HYBRID = 2 };
enum { SLBM_ORDER_CELLS = 0, SLBM_ORDER_VOXELS = 1 };

/* Problem description (Sec. 2 parameters, Sec. 3 geometry). */
typedef struct {
    int32_t nx, ny, nz;        /* voxel box, each >= 1 */
    const uint8_t *flags;      /* HOST, nx*ny*nz flags (0..3), read during create only */
    uint32_t periodic;         /* bit0 x, bit1 y, bit2 z */
    int32_t q;                 /* 19 or 27 */
    int32_t op;                /* SLBM_SRT, SLBM_TRT, SLBM_MRT (D3Q19), SLBM_CM or SLBM_CUMULANT
                                  (D3Q27); MRT, CM and cumulant: sparse and pull layouts */
    double omega_plus;         /* 1/tau in (0, 2) (Eq. 7) */
    double trt_magic;          /* TRT magic parameter Lambda > 0; ignored for SRT */
    double force[3];           /* constant body-force density (Guo) */
    const float *inlet_u;      /* HOST, nullable: 3 floats per inlet voxel, ascending voxel id */
    int64_t n_inlet_u;         /* entries (voxels) in inlet_u; must equal the inlet count */
    double rho_out;            /* pressure-outlet density */
    int32_t storage;           /* SLBM_FP32 / SLBM_FP16 / SLBM_BF16 shifted populations */
    int32_t scale_exp;         /* FP16/BF16: stored value = (f_i - w_i) * 2^scale_exp, |.| <= 40 */
    int32_t layout;            /* SLBM_LAYOUT_SPARSE (the method: one field, AA pattern),
                                  SLBM_LAYOUT_DENSE (comparator) or SLBM_LAYOUT_SPARSE_PULL
                                  (comparison scheme: the same lists, two fields, pull) */
    int32_t order;             /* compacted cell order (Sec. 3.1 numbers cells row-wise):
                                  SLBM_ORDER_LEX, lexicographic with x fastest (default), or
                                  SLBM_ORDER_BRICK8, 8x8x8 bricks in lexicographic brick order
                                  and voxels lexicographic inside each brick (partial bricks at
                                  the high faces); sparse and pull layouts (dense: LEX only) */
} slbm_desc;

/* SLBM_MRT -- multiple-relaxation-time collision (D3Q19 only; the paper
 * lists MRT among its generated operators, Sec. 4, and benchmarks it against
 * SRT/TRT in Sec. 5.1).  Relaxation happens in the orthogonal moment basis of
 * d'Humieres et al. (2002), rows in the order rho, e, eps, jx, qx, jy, qy,
 * jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz, with the Guo
 * force: m* = m - S (m - m_eq) + (I - S/2) M F.  Rates: omega_plus on the
 * five stress moments (the viscosity, Eq. 7) and, until
 * sparse_lbm_set_mrt_rates says otherwise, s_e = 1.19, s_eps = s_pi = 1.4,
 * s_q = 1.2, s_m = 1.98; trt_magic is ignored.  Sparse (AA) and pull
 * layouts, launch variants 0 and 2 with at most 2 cells per thread; no
 * pools. */

/* SLBM_CM, SLBM_CUMULANT -- central-moment and cumulant collisions (D3Q27
 * only; the paper lists both among its generated operators, Sec. 4, and
 * benchmarks them in Sec. 5.1; the cumulants are those of Geier et al.
 * 2015).  Central moments are taken about the Guo velocity u = (j + F/2)/rho;
 * the collision keeps rho, sets the first central moments to +F/2 (the
 * momentum gains F), relaxes the trace of the second ones with the bulk rate
 * towards 3 rho c_s^2 and their deviatoric part with omega_plus (the
 * viscosity, Eq. 7), and the moments of order 3 to 6 with the higher rate:
 * SLBM_CM towards the factorised D3Q27 equilibrium rho prod m(.), m = (1, 0,
 * 1/3); SLBM_CUMULANT relaxes their cumulants (of kappa/rho) towards 0, with
 * the higher rate fixed at 1.  Rates: bulk 1 and higher 1 until
 * sparse_lbm_set_cm_rates says otherwise; trt_magic is ignored.  Launch
 * variants 0 (both steps) and 2 (odd step, 1 or 2 cells); no pools. */

/* SLBM_LAYOUT_SPARSE_PULL -- the two-grid pull scheme the paper compares the
 * AA pattern with (Sec. 5.1, Table 2's pull row): the same compacted cells and
 * canonical pull entries P(i,k), two PDF fields; each step gathers f_i from
 * P(i,k) of one field, collides, and writes the cell's own column of the
 * other (reads Q B_pdf + (Q-1) x 4 index bytes, writes Q B_pdf per cell).  At
 * step 0 the field holds the natural populations; the first step collides in
 * place, so the stored field at step t > 0 is the post-collision C(t-1), and
 * read-outs (macroscopic, reduce) pull it through P.  Walls and periodic
 * boundaries only (SLBM_EUNSUPPORTED with inlet/outlet voxels); one launch
 * shape (set_launch: SLBM_EUNSUPPORTED); no pools, no link codes.
 * get_state/set_state move the stored field of the current step.  Results are
 * bit-identical to the AA layout's at every step. */

/* Optional device allocator.  alloc returns device memory (256-byte aligned)
 * or NULL; free releases it.  Both are called on the creating thread only. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} slbm_allocator;

typedef struct {
    int64_t n_voxels;          /* nx*ny*nz */
    int64_t n_fluid;           /* N_F, fluid cells (Eq. 8 numerator) */
    int64_t stride;            /* S: PDF-list row stride, N_F rounded up to 128 (sparse) or N (dense) */
    int64_t n_bc_links;        /* inlet/outlet links in the index-list */
    int64_t device_bytes;      /* library-owned device memory held by the handle */
    int64_t step;              /* time steps taken (the AA parity is step & 1) */
    int32_t q, op, storage, layout, scale_exp, pad;
} slbm_info;

/* Build a domain from a voxel geometry (Sec. 3.1): copy the flags to the
 * device, compact the fluid cells with a device prefix sum (lexicographic
 * order, bit-identical to a sequential scan), build the pull index-list
 * P(i,k) (Q-1 rows x stride int32; fluid neighbour x_k - c_i -> i*S + its
 * cell, wall -> inverse(i)*S + k, inlet/outlet -> -(b+1) with b the link
 * number in (k, i) order, padding columns -> INT32_MIN) and the boundary-link
 * table, and initialise the rest state (rho = 1, u = 0; all shifted
 * populations zero).  `stream` is a cudaStream_t or NULL.  On success *out
 * owns all device memory of the domain.  Errors: SLBM_EINVAL (bad desc),
 * SLBM_EUNSUPPORTED (Q*S >= 2^31), SLBM_ENOMEM, SLBM_ECUDA. */
slbm_status sparse_lbm_create(const slbm_desc *desc, const slbm_allocator *alloc, void *stream,
                              slbm_t **out);

/* Advance n >= 0 time steps (Eqs. 3-4 fused, AA pattern of Sec. 5.1): step t
 * even -> cell-local collide writing each post-collision PDF into the inverse
 * direction's slot; t odd -> read the index-list, gather through it, collide,
 * scatter back to the slots read.  Asynchronous on the handle's stream.
 * Errors: SLBM_EINVAL (null handle or n < 0), SLBM_ECUDA (a launch failed;
 * the step counter stops at the last step launched).  Faults found by the
 * kernels (checked mode, staging timeouts) are latched on the device and
 * reported by sparse_lbm_device_error. */
slbm_status sparse_lbm_step(slbm_t *h, int32_t n);

/* Same as sparse_lbm_step but replays a CUDA graph holding n launches
 * (captured on first use for each (n, parity) and cached).  Errors as
 * sparse_lbm_step; a failed capture or replay is SLBM_ECUDA. */
slbm_status sparse_lbm_step_graph(slbm_t *h, int32_t n);

/* Macroscopic fields (Eq. 1 with the Guo half-force velocity) of the current
 * state, at either AA parity.  rho: n floats; u: 3 x n floats, component-major
 * (u_x of all cells, then u_y, then u_z).  order SLBM_ORDER_CELLS -> n = N_F
 * in compacted order; SLBM_ORDER_VOXELS -> n = nx*ny*nz, zero off fluid.
 * mem SLBM_MEM_DEVICE -> device pointers, asynchronous; SLBM_MEM_HOST -> host
 * pointers, synchronous.  Either pointer may be NULL. */
slbm_status sparse_lbm_macroscopic(slbm_t *h, float *rho, float *u, int32_t order, int32_t mem);

/* Domain sums in FP64, deterministic (fixed partition and order, independent
 * of launch configuration): out[0] = sum(rho - 1), out[1..3] = sum rho*u,
 * out[4] = sum u_x, over fluid cells.  mem selects a device or host pointer
 * (host: synchronous).  Returns SLBM_EDIVERGED (after writing out) when a sum
 * is not finite. */
slbm_status sparse_lbm_reduce(slbm_t *h, double *out, int32_t mem);

/* Domain sums plus two maxima, for the convergence and stability checks of a
 * solve and for choosing the storage scale of FP16/BF16 populations:
 * out[0..4] = exactly the values of sparse_lbm_reduce (the same bits);
 * out[5] = the largest |f_i - w_i| over the stored populations (shifted,
 * unscaled; every slot of every fluid cell at either AA parity);
 * out[6] = the largest speed |u| (Eq. 1, Guo half-force velocity) over fluid
 * cells.  Both maxima are exact (the order of a maximum does not matter) and
 * a NaN anywhere makes them NaN.  mem as sparse_lbm_reduce; host mode
 * synchronises and returns SLBM_EDIVERGED (after writing out) when a value is
 * not finite or out[6] > 0.3 (beyond the stability bound of the lattice).
 * Device mode writes 7 doubles asynchronously.  Errors: SLBM_EINVAL (NULL
 * argument, bad mem), SLBM_ECUDA. */
slbm_status sparse_lbm_reduce_ext(slbm_t *h, double *out, int32_t mem);

/* Change the storage of the populations in place (the paper's zero-centred
 * storage, Sec. 4, kept in every format): every stored value v of the current
 * format A with scale s_a becomes pack_B(raw_A(v) * 2^(s_b - s_a)) in format
 * `storage` with scale `scale_exp` (ignored for SLBM_FP32, which has none).
 * FP16/BF16 -> FP32 and a power-of-two rescale within FP16/BF16 are exact
 * for values that stay normal numbers; FP32 -> FP16/BF16 rounds to nearest
 * even like every store of the stepping kernels.  The state keeps its step
 * and parity, so stepping continues from it.  A change of element size
 * allocates the new array (through the domain's allocator) before freeing
 * the old one, so a failure leaves the domain unchanged.  Launch shapes are
 * reset to the defaults of the new storage; cached graphs are dropped.
 * Synchronous.  Errors: SLBM_EINVAL (bad storage, scale_exp outside
 * [-40, 40], the domain is a pool member -- slbm_pool_remove it first -- or
 * the converted values would overflow the target format), SLBM_EDIVERGED
 * (a stored value is not finite), SLBM_ENOMEM, SLBM_ECUDA. */
slbm_status sparse_lbm_set_storage(slbm_t *h, int32_t storage, int32_t scale_exp);

/* Set the state to the equilibrium of given fields (Eq. 6): rho (n floats)
 * and u (3 x n, component-major) in cell or voxel order, device or host
 * memory.  NULL rho means 1, NULL u means 0.  Resets the step counter to 0. */
slbm_status sparse_lbm_init_equilibrium(slbm_t *h, const float *rho, const float *u,
                                        int32_t order, int32_t mem);

/* Sizes and state of a domain (the fields of slbm_info) into caller memory.
 * Synchronous, no device access.  Errors: SLBM_EINVAL for a null argument. */
slbm_status sparse_lbm_info(const slbm_t *h, slbm_info *out);

/* Copy the sparse lists to HOST buffers (any pointer may be NULL):
 * cell_voxel[N_F]; index_rows[(Q-1)*S] = the canonical pull entries P(i,k)
 * (row r = direction r+1, values as in sparse_lbm_create); link_cell,
 * link_dir, link_type [n_bc_links]. Synchronous. Sparse layout only.
 * (On the device the list is kept with each non-negative entry's row flipped
 * between i and inverse(i) -- the slot the AA odd step reads; the export
 * flips it back, exactly.) */
slbm_status sparse_lbm_export_lists(const slbm_t *h, int32_t *cell_voxel, int32_t *index_rows,
                                    int32_t *link_cell, int32_t *link_dir, int32_t *link_type);

/* The 16-bit link codes the odd step reads (launch variant 4), to HOST
 * memory: codes [(Q-1) x S] (uint16, row i-1 = direction i) and bases
 * [(S/128) x (Q-1)] (int32, one column base per 128-cell tile and direction).
 * They encode the device's odd-step slot R(i,k) -- the pull entry P(i,k) of
 * Sec. 3.1 with its row flipped between i and inverse(i) -- in 2 bytes.  With
 * b = bases[k/128][i-1]:
 *   b == -1        : the tile-direction's fluid columns span 0xFFFE or
 *                    more; R is read from the int32 list (codes 0xFFFE)
 *   code == 0xFFFE : inlet/outlet link; R is read from the int32 list
 *   code == 0xFFFF : wall (the cell's own slot, R = i*S + k) or padding
 *   otherwise      : fluid neighbour, R = inverse(i)*S + b + code
 * The paper stores 4-byte indices; this encoding is an addition of this
 * library (it halves the index bytes of the odd step).  Builds the codes on
 * first use (as launch variant 4 does).  Either pointer may be NULL.
 * Synchronous.  Sparse layout only. */
slbm_status sparse_lbm_export_codes(slbm_t *h, uint16_t *codes, int32_t *bases);

/* Checkpoint / resume: raw stored PDFs (Q x S elements of the storage type,
 * bytes = Q*S*element size) plus the step counter, to or from HOST memory
 * (caller-owned, `bytes` long).  Synchronous.  A resumed run continues
 * bit-for-bit like an uninterrupted one.  Errors: SLBM_EINVAL (NULL
 * argument, step < 0), SLBM_ECUDA (the copy failed). */
slbm_status sparse_lbm_state_bytes(const slbm_t *h, int64_t *bytes);
slbm_status sparse_lbm_get_state(const slbm_t *h, void *host, int64_t *step);
slbm_status sparse_lbm_set_state(slbm_t *h, const void *host, int64_t step);

/* MRT domains: the relaxation rate of every moment of the basis (19 values
 * in the basis order; the conserved rho, jx, jy, jz entries are ignored; the
 * others must lie in (0, 2)).  The stress entries (9, 11, 13, 14, 15) set
 * the viscosity.  SLBM_EINVAL for non-MRT domains or rates out of range. */
slbm_status sparse_lbm_set_mrt_rates(slbm_t *h, const double *rates);

/* SLBM_CM and SLBM_CUMULANT domains: the relaxation rate of the trace of the
 * second-order central moments (bulk viscosity) and of every moment of
 * order 3 to 6, each in (0, 2].  Cumulant domains take higher == 1 only
 * (SLBM_EUNSUPPORTED otherwise).  SLBM_EINVAL for other domains or rates out
 * of range.  Cached graphs are dropped. */
slbm_status sparse_lbm_set_cm_rates(slbm_t *h, double bulk, double higher);

/* Launch shape used for a parity (0 even, 1 odd), chosen by the autotuner.
 * variant 0: `cells` cells per thread (even 1/2/4 consecutive cells; odd 1/2
 *            cells strided by the block size),
 *            `threads` per block (32..256, multiple of 32);
 * variant 1: persistent CTAs (SMs x resident CTAs) that walk tiles of
 *            `threads` cells (64 or 128) and keep `cells` tiles (2 or 4) of
 *            index-list rows (odd) or PDF rows (even) in flight in shared
 *            memory through asynchronous bulk copies; sparse FP32/FP16 only;
 * variant 2: even step: as variant 0 with 2 or 4 cells per thread that
 *            collide in pairs through the paired FP32 instructions (one
 *            instruction per two cells; the same roundings per cell); MRT:
 *            2 cells.  Odd step: as variant 0 (1 or 2 cells per thread), plus an
 *            asynchronous bulk L2 prefetch of the index-list rows of the block
 *            that will run one residency wave later;
 * variant 3: even step: variant 1 (tile 64 or 128, 2 or 4 stages; sparse
 *            FP32/FP16) with 2 cells per thread collided in pairs as in
 *            variant 2; SRT/TRT.  Odd step: as variant 2, but each thread
 *            re-reads its slots from the list before the scatter instead of
 *            keeping them in registers (domains without inlet/outlet links;
 *            others run variant 2);
 * variant 4: odd step only, as variant 2 (1 or 2 cells per thread), with the
 *            slots read as 16-bit link codes (sparse_lbm_export_codes) and
 *            the L2 prefetch of the codes: 2 instead of 4 index bytes per
 *            link.  The codes ((Q-1) x S x 2 bytes) are built and allocated
 *            on the first selection of this variant (SLBM_ENOMEM if the
 *            allocation fails);
 * variant 5: SRT/TRT: odd step only, as variant 2 with 1 cell per thread,
 *            the kernel held to 64 registers a thread (more resident warps,
 *            some registers spilled to L1).  MRT, central-moment and
 *            cumulant domains: both steps, 128 x 1 (odd with the L2 index
 *            prefetch), the kernels held to five resident blocks a
 *            multiprocessor (at most 102 registers a thread);
 * variant 6: odd step only, sparse SRT/TRT: 128 threads (one tile of cells)
 *            and `cells` (2..4) shared-memory stages: a producer warp copies
 *            each tile's 16-bit window codes, own rows and gather windows in
 *            with the bulk-copy engine while four warps compute the previous
 *            tile from shared memory.  The window table and codes
 *            ((S / 128) x (Q-1) x 16 + (Q-1) x S x 2 bytes) are built on the
 *            first selection (SLBM_ENOMEM if the allocation fails).
 * Operators: MRT, central-moment and cumulant domains run even variants 0
 * and 5 (MRT also 2) with 1 or 2 cells per thread and odd variants 0, 2, 3
 * (no links) and 5; the rest SLBM_EUNSUPPORTED.  The hybrid cell order runs
 * one odd shape: 128 x 1, variant 2 (the full bricks by their own kernel).
 * Defaults: even variant 2, 64 x 4 (FP16 D3Q27 with inlet/outlet links:
 * variant 1, tile 128, 2 stages; FP32 MRT: variant 2, 64 x 2; FP16 MRT and
 * BF16: variant 0, 64 x 2; central-moment and cumulant: variant 0, 64 x 1,
 * 16-bit storage 64 x 2); odd variant 2 (D3Q19: FP32 128 x 2, or 128 x 1
 * with links, FP16 256 x 1; D3Q27 without links: FP32 256 x 1, FP16
 * 256 x 2; D3Q27 with links: FP32 64 x 1, FP16 variant 5, 128 x 1; BF16,
 * the pull and dense layouts 128 x 1; MRT: variant 5, 128 x 1;
 * central-moment and cumulant: 256 x 1).  Results are bit-for-bit the same
 * for every shape. */
slbm_status sparse_lbm_set_launch(slbm_t *h, int32_t parity, int32_t threads, int32_t cells, int32_t variant);

/* Kernel check mode: 1 = odd-step gathers bounds-check every slot and latch
 * SLBM_EDEVICE instead of touching memory out of range; 0 = fast path. */
slbm_status sparse_lbm_set_checked(slbm_t *h, int32_t on);

/* Latched device error (0 none), synchronising the stream. Clears it.
 * Returns SLBM_EDEVICE when a code was latched (also written to *code),
 * SLBM_EINVAL for a NULL argument, SLBM_ECUDA if the synchronisation fails. */
slbm_status sparse_lbm_device_error(slbm_t *h, int32_t *code);

/* Release everything (a pool that still holds the domain loses it as a
 * member, after its queued work); NULL is a no-op. */
void sparse_lbm_free(slbm_t *h);

/* Largest voxel count sparse_lbm_compact_noalloc accepts (65536 scan tiles of
 * 4096 voxels; e.g. a 1024 x 512 x 512 box). */
#define SLBM_NOALLOC_MAX_VOXELS 268435456

/* Fluid-cell compaction that allocates nothing (the paper has no counterpart;
 * it is a service for callers that cannot let a library allocate).
 *
 * Who needs it: callers that own every byte of device memory themselves -- a
 * framework that reserves one arena up front and forbids other allocations,
 * or a latency-critical loop where cudaMalloc/cudaFree, which may synchronise
 * the whole device, are not acceptable.  They pass device buffers in and get
 * results out; the call makes no cudaMalloc, cudaFree or other allocating
 * library call.
 *
 * What it computes: the compaction in the
 * lexicographic order SLBM_ORDER_LEX that sparse_lbm_create uses: cell_id[v] = rank of voxel v
 * among fluid voxels (flag 0) in ascending voxel id, or -1; cell_voxel[k] = voxel id of fluid cell k; *n_fluid = count.
 * All pointers are DEVICE pointers: flags[n_voxels] (uint8), cell_id[n_voxels],
 * cell_voxel[capacity >= number of fluid voxels], n_fluid[1] (int32).  The work
 * is enqueued on `stream` (cudaStream_t or NULL) and the call returns without
 * waiting; read *n_fluid after synchronising the stream.
 *
 * Scratch: the scan's per-tile totals live in one fixed device array inside
 * the library (256 KiB), which every GPU that loads the library holds until
 * the process exits.  All calls share it and it keeps the last call's
 * contents; each call overwrites what it reads first.  Calls that overlap on
 * the GPU (e.g. on two streams at once) race on it: serialise them.  Every
 * call made outside a stream capture looks up the array's device address on
 * the current device (so a device reset that reloads the library's module is
 * followed); a call made while `stream` is being captured uses the address
 * that the last call outside capture found on that device, so make one call
 * on the device before any capture (SLBM_ECUDA otherwise).
 *
 * Errors: SLBM_EINVAL if n_voxels < 0, n_voxels > SLBM_NOALLOC_MAX_VOXELS or a
 * needed pointer is NULL (nothing is launched); SLBM_ECUDA if the device or a
 * launch fails. */
slbm_status sparse_lbm_compact_noalloc(const uint8_t *flags, int64_t n_voxels, int32_t *cell_id,
                                       int32_t *cell_voxel, int32_t *n_fluid, void *stream);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *sparse_lbm_last_error(void);

/* ---- batching: many domains stepped by one persistent kernel ----------------
 * A pool steps many member domains together.  Members below a cell threshold
 * (slbm_pool_set_split) are batched: their compacted cell lists are
 * concatenated through a device domain table (per-domain tile offset, stride,
 * parity, rates, force, link maps) and one launch per time step covers a
 * group of them (slbm_pool_set_group_bytes), each at its own AA parity
 * (Sec. 5.1).  Larger members run their own single-domain kernels in the same
 * sequence, optionally on extra streams (slbm_pool_set_streams).  Members keep
 * their own memory and handles; all must share q and storage and use the
 * sparse layout with SRT/TRT.  The per-cell arithmetic is the single-domain
 * kernels', so a member's state evolves bit for bit as it would alone.  Pool
 * work runs on the pool's stream: synchronise it (any pool call that returns
 * host data does) before using a member handle directly. */
/* A pool for members of stencil q (19 | 27) and storage (as slbm_desc) with
 * `capacity` slots (1..65536); `stream` is a cudaStream_t or NULL.  Errors:
 * SLBM_EINVAL (bad q, storage or capacity, NULL out), SLBM_ENOMEM,
 * SLBM_ECUDA (no device). */
slbm_status slbm_pool_create(int32_t q, int32_t storage, int32_t capacity, void *stream,
                             slbm_pool_t **out);
/* Add a domain (not owned by the pool) to a free slot, written to *slot.
 * Errors: SLBM_EINVAL (NULL argument, q or storage differing from the pool's,
 * already a member), SLBM_EUNSUPPORTED (not the sparse layout, or MRT),
 * SLBM_ENOMEM (no free slot). */
slbm_status slbm_pool_add(slbm_pool_t *p, slbm_t *h, int32_t *slot);
/* Remove a member after its queued pool work has finished (synchronises). */
slbm_status slbm_pool_remove(slbm_pool_t *p, int32_t slot);
/* k >= 0 steps on every member (each at its own parity); use_graph != 0
 * replays CUDA graphs: one of the batched groups' k launches (captured again
 * when the batched table changes) and each large member's own graph of k
 * steps (kept across membership changes). */
slbm_status slbm_pool_step(slbm_pool_t *p, int32_t k, int32_t use_graph);
/* out: 5 doubles per slot (capacity x 5, layout as sparse_lbm_reduce), device
 * or host; free slots are zero.  Bit-identical to sparse_lbm_reduce of each
 * member.  Host mode returns SLBM_EABORTED if an abort was raised since the
 * last clear. */
slbm_status slbm_pool_reduce(slbm_pool_t *p, double *out, int32_t mem);
/* As slbm_pool_reduce with sparse_lbm_reduce_ext's 7 values per slot
 * (capacity x 7 doubles; free slots are zero); host mode returns
 * SLBM_EABORTED like slbm_pool_reduce and does not test the values. */
slbm_status slbm_pool_reduce_ext(slbm_pool_t *p, double *out, int32_t mem);
/* Launch variant.  ctas_per_sm == 0 (default): tile grid -- one CTA of 128
 * threads per tile of the concatenated cell lists (256-cell tiles for the even
 * step, 128-cell tiles for the odd step); each launch carries its group's
 * member table (up to 256 members) as a kernel parameter, rebuilt on the host
 * when the membership changes (threads is ignored).  ctas_per_sm > 0:
 * persistent walker with `threads` cells per tile (32..128, multiple of 32)
 * and at most ctas_per_sm CTAs per SM. */
slbm_status slbm_pool_set_launch(slbm_pool_t *p, int32_t threads, int32_t ctas_per_sm);
/* Members with at least split_cells fluid cells (default 524288) are stepped
 * by their own single-domain kernels inside the pool's launch sequence (and
 * graph); smaller members share the batched launch.  0 = batch every member.
 * Applies to the tile-grid variant. */
slbm_status slbm_pool_set_split(slbm_pool_t *p, int64_t split_cells);
/* Launch order of the tile-grid variant.  The batched members are cut, in
 * slot order, into groups whose state + index + link-map bytes sum to at most
 * `bytes` (default 48 MiB; a member larger than that is a group of its own);
 * one slbm_pool_step(k) runs group after group, each for all k steps, then
 * each large member for its k steps.  A group that fits in L2 streams its k
 * steps from L2.  0 = one group of all batched members (every launch covers
 * all of them).  Members are independent: the order changes no result. */
slbm_status slbm_pool_set_group_bytes(slbm_pool_t *p, int64_t bytes);
/* Streams of a graph step (use_graph != 0, tile-grid variant): n == 1
 * (default) runs everything in order on the pool's stream.  n > 1 (at most
 * 16) forks n - 1 extra streams, owned by the pool, from the pool's stream:
 * the batched groups stay on the pool's stream, each large member goes to the
 * stream with the fewest fluid cells queued in this step, and the pool's
 * stream waits for all of them before the step returns.  Work on the pool's
 * stream after the step (reduce, remove, free) sees every member finished.
 * Members are independent: the spread changes no result. */
slbm_status slbm_pool_set_streams(slbm_pool_t *p, int32_t n);
/* raise != 0: set the host-mapped abort word; running and queued batched pool
 * launches stop at their next tile (members stepped by their own kernels
 * finish theirs) and the members' states are left part-way through a step
 * (restore them from a checkpoint).  raise == 0: wait for the pool's
 * stream, then clear the word and the latched status. */
slbm_status slbm_pool_abort(slbm_pool_t *p, int32_t raise);
/* Wait for the pool's queued work, then release the pool (not its members,
 * which stay valid and are no longer pool members); NULL is a no-op. */
void slbm_pool_free(slbm_pool_t *p);

#ifdef __cplusplus
}
#endif
#endif /* SPARSE_LBM_H */
