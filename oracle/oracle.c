/*
 * oracle.c -- plain, slow, FP64 CPU lattice Boltzmann reference.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the graft smoke check and the benchmark's
 * CPU-baseline arm do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper Sec. 2, Eqs. 1-6, and Sec. 3.1 for the lists):
 *   - the macroscopic moments rho = sum f_i, rho*u = sum c_i f_i        (Eq. 1)
 *   - collide  f~_i = f_i + Omega_i                                      (Eq. 3)
 *     with SRT  Omega_i = -omega (f_i - f_i^eq)                           (Eq. 5)
 *     or TRT (two relaxation rates on the even/odd parts; textbook form,
 *     the paper names TRT in Sec. 4 and cites the LBM textbook for it),
 *     or MRT (D3Q19: relaxation in the orthogonal moment space of
 *     d'Humieres et al. 2002, one rate per moment; the paper lists MRT among
 *     its generated operators, Sec. 4, and benchmarks it in Sec. 5.1),
 *     second-order equilibrium f_i^eq                                     (Eq. 6)
 *     and a Guo body-force source (the paper says only "a force model",
 *     Sec. 4; the Guo form is our reading)
 *   - stream   f_i(x + c_i, t+1) = f~_i(x, t)                             (Eq. 4)
 *     as a two-grid PUSH over a dense, direct-addressed box (Sec. 3),
 *     with halfway bounce-back at walls (Sec. 3.1.1), periodic wrap,
 *     a Ladd moving-wall (UBB) inlet and an anti-bounce-back pressure outlet
 *     whose equilibrium uses the boundary cell's own velocity (both textbook
 *     forms; the paper only says such boundaries exist, Sec. 3.1.1).
 *   - its own sparse indexing (Sec. 3.1): the compacted fluid-cell order
 *     (lexicographic, x fastest), the pull index-list P(i,k) with no-slip
 *     links pointing at the same cell's inverse direction and periodic links
 *     wrapped, and a sparse two-grid pull stepper that uses the same per-cell
 *     arithmetic as the dense stepper.
 *
 * PDFs are stored unshifted (f, not f - w) in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_FLUID = 0, ORC_WALL = 1, ORC_INLET = 2, ORC_OUTLET = 3 };
enum { ORC_SRT = 0, ORC_TRT = 1, ORC_MRT = 2, ORC_CM = 3, ORC_CUM = 4 };

/* Velocity set, directions written out one by one (D3Q19 is the first 19
 * rows of D3Q27).  Ordering convention: rest, then the six axis directions,
 * then the twelve edge directions, then the eight corners, each followed
 * immediately by its inverse. */
static const int VEL[27][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1},
    {1, 0, -1},  {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},
    {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1},
    {-1, 1, 1},  {1, -1, -1}};

typedef struct {
    int32_t nx, ny, nz;
    const uint8_t *flags;      /* nx*ny*nz, x fastest */
    uint32_t periodic;         /* bit0 x, bit1 y, bit2 z */
    int32_t q;                 /* 19 or 27 */
    int32_t op;                /* ORC_SRT or ORC_TRT */
    double omega_plus;         /* 1/tau */
    double omega_minus;        /* TRT odd rate (ignored for SRT) */
    double force[3];           /* body-force density (Guo) */
    const double *inlet_u;     /* 3 per inlet voxel, ascending voxel order; may be NULL */
    double rho_out;            /* outlet density */
    double mrt_s[19];          /* ORC_MRT (D3Q19): relaxation rate of each moment of the basis below */
    int32_t order;             /* cell order: 0 lexicographic, 1 brick-8, 2 full bricks first (orc_compact) */
    double cm_bulk;            /* ORC_CM / ORC_CUM (D3Q27): rate of the trace of the second-order moments */
    double cm_high;            /* ORC_CM / ORC_CUM: rate of every moment (cumulant) of order 3..6 */
} orc_problem;

/* ---------------------------------------------------------------- stencil */

/* Weight of a direction from its squared length (D3Q19 / D3Q27 textbook
 * values). */
static double weight(int q, int i) {
    int n2 = VEL[i][0] * VEL[i][0] + VEL[i][1] * VEL[i][1] + VEL[i][2] * VEL[i][2];
    if (q == 19) {
        if (n2 == 0) return 1.0 / 3.0;
        if (n2 == 1) return 1.0 / 18.0;
        return 1.0 / 36.0;
    }
    if (n2 == 0) return 8.0 / 27.0;
    if (n2 == 1) return 2.0 / 27.0;
    if (n2 == 2) return 1.0 / 54.0;
    return 1.0 / 216.0;
}

/* Inverse direction, found by searching the table for -c_i. */
static int inverse(int q, int i) {
    for (int j = 0; j < q; ++j)
        if (VEL[j][0] == -VEL[i][0] && VEL[j][1] == -VEL[i][1] && VEL[j][2] == -VEL[i][2])
            return j;
    return -1;
}

int orc_stencil(int q, int32_t *c, double *w, int32_t *inv) {
    if (q != 19 && q != 27) return -1;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = VEL[i][a];
        w[i] = weight(q, i);
        inv[i] = inverse(q, i);
    }
    return 0;
}

/* ---------------------------------------------------- per-cell arithmetic */

/* Eq. 6, c_s^2 = 1/3. */
void orc_equilibrium(int q, double rho, const double u[3], double *feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < q; ++i) {
        double cu = VEL[i][0] * u[0] + VEL[i][1] * u[1] + VEL[i][2] * u[2];
        feq[i] = weight(q, i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Guo source S_i = w_i [ 3 (c_i - u) + 9 (c_i . u) c_i ] . F  (without the
 * (1 - omega/2) prefactor, which the collision applies). */
void orc_guo_source(int q, const double u[3], const double F[3], double *S) {
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    for (int i = 0; i < q; ++i) {
        double cu = VEL[i][0] * u[0] + VEL[i][1] * u[1] + VEL[i][2] * u[2];
        double cF = VEL[i][0] * F[0] + VEL[i][1] * F[1] + VEL[i][2] * F[2];
        S[i] = weight(q, i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
    }
}

/* Eq. 1 with the Guo half-force velocity: rho = sum f, u = (sum c f + F/2)/rho. */
void orc_moments(int q, const double *f, const double F[3], double *rho_out, double u_out[3]) {
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += VEL[i][a] * f[i];
    }
    *rho_out = rho;
    for (int a = 0; a < 3; ++a) u_out[a] = (j[a] + 0.5 * F[a]) / rho;
}

/* D3Q19 moment basis of d'Humieres, Ginzburg, Krafczyk, Lallemand, Luo
 * (2002), row a evaluated at velocity c = (x, y, z), |c|^2 = n:
 *   0 rho 1              1 e  19n - 30          2 eps (21n^2 - 53n + 24)/2
 *   3 jx  x              4 qx (5n - 9) x        5 jy  y     6 qy (5n - 9) y
 *   7 jz  z              8 qz (5n - 9) z
 *   9 3pxx 3x^2 - n      10 3pixx (3n - 5)(3x^2 - n)
 *   11 pww y^2 - z^2     12 piww (3n - 5)(y^2 - z^2)
 *   13 pxy xy   14 pyz yz   15 pxz xz
 *   16 mx x(y^2 - z^2)   17 my y(z^2 - x^2)   18 mz z(x^2 - y^2)
 * The rows are mutually orthogonal over the 19 velocities (a test checks
 * it), so M^-1 = M^T diag(1 / |row a|^2). */
static double mrt_row(int a, int i) {
    double x = VEL[i][0], y = VEL[i][1], z = VEL[i][2], n = x * x + y * y + z * z;
    switch (a) {
        case 0: return 1.0;
        case 1: return 19.0 * n - 30.0;
        case 2: return (21.0 * n * n - 53.0 * n + 24.0) / 2.0;
        case 3: return x;
        case 4: return (5.0 * n - 9.0) * x;
        case 5: return y;
        case 6: return (5.0 * n - 9.0) * y;
        case 7: return z;
        case 8: return (5.0 * n - 9.0) * z;
        case 9: return 3.0 * x * x - n;
        case 10: return (3.0 * n - 5.0) * (3.0 * x * x - n);
        case 11: return y * y - z * z;
        case 12: return (3.0 * n - 5.0) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return x * (y * y - z * z);
        case 17: return y * (z * z - x * x);
        default: return z * (x * x - y * y);
    }
}

/* The 19 x 19 matrix M[a][i] (row-major), for the tests. */
void orc_mrt_matrix(double *M) {
    for (int a = 0; a < 19; ++a)
        for (int i = 0; i < 19; ++i) M[a * 19 + i] = mrt_row(a, i);
}

/* MRT collision in moment space (D3Q19):
 *   m = M f, m_eq = M f_eq, m_F = M S (Guo source)
 *   m*_a = m_a - s_a (m_a - m_eq_a) + (1 - s_a/2) m_F_a
 *   f* = M^-1 m* */
static void collide_mrt(const orc_problem *p, const double *f, const double *feq, const double *S, double *fs) {
    double m[19], me[19], mf[19], nrm[19];
    for (int a = 0; a < 19; ++a) {
        m[a] = me[a] = mf[a] = nrm[a] = 0.0;
        for (int i = 0; i < 19; ++i) {
            double r = mrt_row(a, i);
            m[a] += r * f[i];
            me[a] += r * feq[i];
            mf[a] += r * S[i];
            nrm[a] += r * r;
        }
        double s = p->mrt_s[a];
        m[a] = m[a] - s * (m[a] - me[a]) + (1.0 - 0.5 * s) * mf[a];
    }
    for (int i = 0; i < 19; ++i) {
        double v = 0.0;
        for (int a = 0; a < 19; ++a) v += mrt_row(a, i) * m[a] / nrm[a];
        fs[i] = v;
    }
}

/* ------------------------------------------- central-moment and cumulant
 * collisions (D3Q27; Sec. 4 lists both among the generated operators, Sec.
 * 5.1 benchmarks them; definitions: central moments about the Guo velocity
 * u, cumulants of Geier et al. 2015, both with the density factored out of
 * orders >= 2).
 *
 * Central moments: kap[a + 3b + 9c] = sum_i f_i (cx_i - ux)^a (cy_i - uy)^b
 * (cz_i - uz)^c, a, b, c in {0, 1, 2}.  With u = (j + F/2)/rho the first
 * ones are -F/2.  The collision keeps kap_000 = rho, sets the first ones to
 * +F/2 (the momentum gains F), relaxes the second ones -- the trace with
 * cm_bulk towards 3 rho c_s^2, the two normal differences and the three
 * off-diagonal ones with omega_plus towards 0 -- and the moments of order
 * 3..6 with cm_high: towards rho * prod m(.) with m(0) = 1, m(1) = 0,
 * m(2) = 1/3 (the factorised equilibrium of D3Q27) for ORC_CM; for ORC_CUM
 * their cumulants (of the normalised central moments kap/rho, the first
 * ones taken as zero) towards 0.  Back to f through the inverse of the
 * central-moment map. */
static double ipow3(double x, int n) { return n == 0 ? 1.0 : (n == 1 ? x : x * x); }

void orc_central_moments(const double *f, const double u[3], double *kap) {
    for (int m = 0; m < 27; ++m) {
        int a = m % 3, b = (m / 3) % 3, c = m / 9;
        double s = 0.0;
        for (int i = 0; i < 27; ++i)
            s += f[i] * ipow3(VEL[i][0] - u[0], a) * ipow3(VEL[i][1] - u[1], b) * ipow3(VEL[i][2] - u[2], c);
        kap[m] = s;
    }
}

/* Inverse of the 3 x 3 map k_alpha = sum_c (c - u)^alpha f_c, c = -1, 0, 1,
 * by Gauss-Jordan elimination with partial pivoting: Ai[c + 1][alpha]. */
static void inverse_1d(double u, double Ai[3][3]) {
    double A[3][6];
    for (int al = 0; al < 3; ++al)
        for (int c = 0; c < 3; ++c) {
            A[al][c] = ipow3((double)(c - 1) - u, al);
            A[al][3 + c] = al == c ? 1.0 : 0.0;
        }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        for (int k = 0; k < 6; ++k) {
            double t = A[col][k];
            A[col][k] = A[piv][k];
            A[piv][k] = t;
        }
        double d = A[col][col];
        for (int k = 0; k < 6; ++k) A[col][k] /= d;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            double e = A[r][col];
            for (int k = 0; k < 6; ++k) A[r][k] -= e * A[col][k];
        }
    }
    /* A^-1 maps (k_0, k_1, k_2) to (f_-1, f_0, f_1): its rows are indexed by c */
    for (int c = 0; c < 3; ++c)
        for (int al = 0; al < 3; ++al) Ai[c][al] = A[c][3 + al];
}

void orc_from_central(const double *kap, const double u[3], double *f) {
    double X[3][3], Y[3][3], Z[3][3];
    inverse_1d(u[0], X);
    inverse_1d(u[1], Y);
    inverse_1d(u[2], Z);
    for (int i = 0; i < 27; ++i) {
        int px = VEL[i][0] + 1, py = VEL[i][1] + 1, pz = VEL[i][2] + 1;
        double s = 0.0;
        for (int m = 0; m < 27; ++m) s += X[px][m % 3] * Y[py][(m / 3) % 3] * Z[pz][m / 9] * kap[m];
        f[i] = s;
    }
}

/* Moment / cumulant conversion by the set-partition formulas, for the
 * multiset of axes of index m (x a times, y b times, z c times, n <= 6):
 *   cumulant = sum over partitions pi of (-1)^(|pi|-1) (|pi|-1)! prod_B mom(B)
 *   moment   = sum over partitions pi of prod_B cum(B)
 * where a block's value is that of its own axis multiset; blocks of one
 * element are zero (zero mean), so those partitions are left out.  The
 * partitions of each index are enumerated once (restricted growth strings)
 * into a table when the library is loaded. */
#define PART_MAX 64
typedef struct {
    int n_part;
    int n_blk[PART_MAX];
    int blk[PART_MAX][3];          /* at most 3 blocks of >= 2 elements among 6 */
} part_table;
static part_table PARTS[27];

static void enumerate_partitions(int m, const int *axis, int n, int *label, int pos, int nblk) {
    if (pos == n) {
        int idx[6], size[6];
        for (int b = 0; b < nblk; ++b) idx[b] = size[b] = 0;
        for (int e = 0; e < n; ++e) {
            static const int W[3] = {1, 3, 9};
            idx[label[e]] += W[axis[e]];
            ++size[label[e]];
        }
        for (int b = 0; b < nblk; ++b)
            if (size[b] == 1) return;
        part_table *t = &PARTS[m];
        t->n_blk[t->n_part] = nblk;
        for (int b = 0; b < nblk; ++b) t->blk[t->n_part][b] = idx[b];
        ++t->n_part;
        return;
    }
    for (int b = 0; b <= nblk; ++b) {
        label[pos] = b;
        enumerate_partitions(m, axis, n, label, pos + 1, b == nblk ? nblk + 1 : nblk);
    }
}

__attribute__((constructor)) static void build_partition_tables(void) {
    for (int m = 0; m < 27; ++m) {
        int axis[6], label[6], n = 0;
        int cnt[3] = {m % 3, (m / 3) % 3, m / 9};
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < cnt[a]; ++k) axis[n++] = a;
        PARTS[m].n_part = 0;
        if (n >= 2) enumerate_partitions(m, axis, n, label, 0, 0);
    }
}

static double convert(int m, const double *val, int to_cumulant) {
    const part_table *t = &PARTS[m];
    double s = 0.0;
    for (int q = 0; q < t->n_part; ++q) {
        double prod = 1.0;
        for (int b = 0; b < t->n_blk[q]; ++b) prod *= val[t->blk[q][b]];
        if (to_cumulant) {
            double fact = 1.0;
            for (int k = 2; k < t->n_blk[q]; ++k) fact *= k;
            prod *= ((t->n_blk[q] - 1) % 2 ? -1.0 : 1.0) * fact;
        }
        s += prod;
    }
    return s;
}

static int order_of(int m) { return m % 3 + (m / 3) % 3 + m / 9; }

/* Normalised cumulants of orders >= 2 of f about the Guo velocity (orders 0
 * and 1 returned as 0), for the tests. */
void orc_cumulants(const orc_problem *p, const double *f, double *cum) {
    double rho, u[3], kap[27], mom[27];
    orc_moments(27, f, p->force, &rho, u);
    orc_central_moments(f, u, kap);
    for (int m = 0; m < 27; ++m) mom[m] = order_of(m) >= 2 ? kap[m] / rho : 0.0;
    for (int m = 0; m < 27; ++m) cum[m] = order_of(m) >= 2 ? convert(m, mom, 1) : 0.0;
}

/* Second-order relaxation of the moment-indexed array v (index a + 3b +
 * 9c): the normal entries v[2] (xx), v[6] (yy), v[18] (zz) as their trace,
 * relaxed with wb towards 3 eq, and the differences xx - yy, xx - zz,
 * relaxed with w towards 0; the off-diagonal v[4] (xy), v[10] (xz), v[12]
 * (yz) with w towards 0. */
static void relax_second(double *v, double eq, double w, double wb) {
    const int XX = 2, YY = 6, ZZ = 18, XY = 4, XZ = 10, YZ = 12;
    double T = v[XX] + v[YY] + v[ZZ], D1 = v[XX] - v[YY], D2 = v[XX] - v[ZZ];
    T -= wb * (T - 3.0 * eq);
    D1 *= 1.0 - w;
    D2 *= 1.0 - w;
    v[XX] = (T + D1 + D2) / 3.0;
    v[YY] = (T - 2.0 * D1 + D2) / 3.0;
    v[ZZ] = (T + D1 - 2.0 * D2) / 3.0;
    v[XY] *= 1.0 - w;
    v[XZ] *= 1.0 - w;
    v[YZ] *= 1.0 - w;
}

static void collide_central(const orc_problem *p, const double *f, double *fs) {
    double rho, u[3], kap[27];
    orc_moments(27, f, p->force, &rho, u);
    orc_central_moments(f, u, kap);
    double w = p->omega_plus, wb = p->cm_bulk, wh = p->cm_high;
    if (p->op == ORC_CM) {
        relax_second(kap, rho / 3.0, w, wb);
        for (int m = 0; m < 27; ++m) {
            if (order_of(m) < 3) continue;
            double eq = rho;
            int cnt[3] = {m % 3, (m / 3) % 3, m / 9};
            for (int a = 0; a < 3; ++a) eq *= cnt[a] == 0 ? 1.0 : (cnt[a] == 1 ? 0.0 : 1.0 / 3.0);
            kap[m] -= wh * (kap[m] - eq);
        }
    } else {
        double mom[27], cum[27], post[27];
        for (int m = 0; m < 27; ++m) mom[m] = order_of(m) >= 2 ? kap[m] / rho : 0.0;
        for (int m = 0; m < 27; ++m) cum[m] = order_of(m) >= 2 ? convert(m, mom, 1) : 0.0;
        relax_second(cum, 1.0 / 3.0, w, wb);
        for (int m = 0; m < 27; ++m)
            if (order_of(m) >= 3) cum[m] *= 1.0 - wh;
        for (int m = 0; m < 27; ++m) post[m] = order_of(m) >= 2 ? convert(m, cum, 0) : 0.0;
        for (int m = 0; m < 27; ++m)
            if (order_of(m) >= 2) kap[m] = rho * post[m];
    }
    kap[0] = rho;
    kap[1] = 0.5 * p->force[0];
    kap[3] = 0.5 * p->force[1];
    kap[9] = 0.5 * p->force[2];
    orc_from_central(kap, u, fs);
}

/* One cell's collision (Eq. 3 with Eq. 5, TRT or MRT): f -> fs. */
void orc_collide(const orc_problem *p, const double *f, double *fs) {
    int q = p->q;
    double rho, u[3], feq[27], S[27];
    orc_moments(q, f, p->force, &rho, u);
    orc_equilibrium(q, rho, u, feq);
    orc_guo_source(q, u, p->force, S);
    if (p->op == ORC_CM || p->op == ORC_CUM) {
        collide_central(p, f, fs);
        return;
    }
    if (p->op == ORC_MRT) {
        collide_mrt(p, f, feq, S, fs);
        return;
    }
    double wp = p->omega_plus;
    if (p->op == ORC_SRT) {
        for (int i = 0; i < q; ++i)
            fs[i] = f[i] - wp * (f[i] - feq[i]) + (1.0 - 0.5 * wp) * S[i];
        return;
    }
    double wm = p->omega_minus;
    for (int i = 0; i < q; ++i) {
        int b = inverse(q, i);
        double fp = 0.5 * (f[i] + f[b]), fm = 0.5 * (f[i] - f[b]);
        double ep = 0.5 * (feq[i] + feq[b]), em = 0.5 * (feq[i] - feq[b]);
        double sp = 0.5 * (S[i] + S[b]), sm = 0.5 * (S[i] - S[b]);
        fs[i] = f[i] - wp * (fp - ep) - wm * (fm - em) + (1.0 - 0.5 * wp) * sp +
                (1.0 - 0.5 * wm) * sm;
    }
}

/* Value a boundary link hands to the fluid cell: the PDF of direction r
 * that re-enters the cell after its own post-collision PDF of direction
 * inverse(r) (value `src`) hit the boundary voxel.  `uc` is the cell's own
 * velocity (Eq. 1 with the Guo half force) at the collision that produced
 * `src`.
 *   wall:   src                                        (halfway bounce-back)
 *   inlet:  src + 6 w_r rho0 (c_r . u_w), rho0 = 1      (Ladd moving wall)
 *   outlet: -src + 2 w_r rho_out (1 + 4.5 (c_r . uc)^2 - 1.5 uc . uc)
 *           (anti-bounce-back towards the even part of the equilibrium at the
 *           outlet density and the cell's velocity) */
static double bc_value(const orc_problem *p, int type, double src, int r, const double *uw, const double *uc) {
    double w = weight(p->q, r);
    if (type == ORC_INLET) {
        double cu = VEL[r][0] * uw[0] + VEL[r][1] * uw[1] + VEL[r][2] * uw[2];
        return src + 6.0 * w * cu;
    }
    if (type == ORC_OUTLET) {
        double cu = VEL[r][0] * uc[0] + VEL[r][1] * uc[1] + VEL[r][2] * uc[2];
        double uu = uc[0] * uc[0] + uc[1] * uc[1] + uc[2] * uc[2];
        return -src + 2.0 * w * p->rho_out * (1.0 + 4.5 * cu * cu - 1.5 * uu);
    }
    return src;
}

/* ------------------------------------------------------------ geometry */

static int64_t nvox(const orc_problem *p) { return (int64_t)p->nx * p->ny * p->nz; }

/* Neighbour voxel of (x,y,z) displaced by d: returns its linear id, or -1
 * when it leaves the box through a non-periodic face (treated as a wall). */
static int64_t neighbour(const orc_problem *p, int x, int y, int z, int dx, int dy, int dz) {
    int n[3] = {x + dx, y + dy, z + dz};
    int dim[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 0 || n[a] >= dim[a]) {
            if (!(p->periodic >> a & 1u)) return -1;
            n[a] = (n[a] + dim[a]) % dim[a];
        }
    }
    return (int64_t)n[0] + (int64_t)p->nx * ((int64_t)n[1] + (int64_t)p->ny * n[2]);
}

static int type_of(const orc_problem *p, int64_t v) { return v < 0 ? ORC_WALL : p->flags[v]; }

/* Rank of each inlet voxel among inlet voxels in ascending voxel order. */
static int64_t *inlet_rank(const orc_problem *p) {
    int64_t n = nvox(p);
    int64_t *r = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t c = 0;
    for (int64_t v = 0; v < n; ++v) r[v] = (p->flags[v] == ORC_INLET) ? c++ : -1;
    return r;
}

static const double ZERO3[3] = {0.0, 0.0, 0.0};
static const double *inlet_velocity(const orc_problem *p, const int64_t *rank, int64_t v) {
    if (!p->inlet_u || v < 0 || rank[v] < 0) return ZERO3;
    return p->inlet_u + 3 * rank[v];
}

/* ------------------------------------------------------- dense stepping */

/* f: Q x N array (direction-major), all voxels; only fluid voxels are
 * meaningful.  Initialises fluid voxels to f^eq(rho, u) (rho, u per voxel;
 * NULL means the rest state rho = 1, u = 0). */
void orc_dense_init(const orc_problem *p, const double *rho, const double *u, double *f) {
    int64_t n = nvox(p);
    for (int64_t v = 0; v < n; ++v) {
        double r = rho ? rho[v] : 1.0;
        double uv[3] = {u ? u[3 * v] : 0.0, u ? u[3 * v + 1] : 0.0, u ? u[3 * v + 2] : 0.0};
        double feq[27];
        orc_equilibrium(p->q, r, uv, feq);
        for (int i = 0; i < p->q; ++i) f[(int64_t)i * n + v] = p->flags[v] == ORC_FLUID ? feq[i] : 0.0;
    }
}

/* `steps` two-grid push steps: collide every fluid voxel of A, push each
 * post-collision PDF to its neighbour in B (or reflect it at a boundary),
 * then swap.  Result is left in f. */
int orc_dense_run(const orc_problem *p, double *f, int steps) {
    int64_t n = nvox(p);
    int q = p->q;
    double *B = (double *)malloc(sizeof(double) * (size_t)(q * n > 0 ? q * n : 1));
    if (!B) return -1;
    memcpy(B, f, sizeof(double) * (size_t)(q * n));
    int64_t *rank = inlet_rank(p);
    double *A = f;
    for (int t = 0; t < steps; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < n; ++v) {
            if (p->flags[v] != ORC_FLUID) continue;
            int x = (int)(v % p->nx), y = (int)((v / p->nx) % p->ny), z = (int)(v / ((int64_t)p->nx * p->ny));
            double fl[27], fs[27], rho, uc[3];
            for (int i = 0; i < q; ++i) fl[i] = A[(int64_t)i * n + v];
            orc_moments(q, fl, p->force, &rho, uc);
            orc_collide(p, fl, fs);
            for (int i = 0; i < q; ++i) {
                int64_t nb = neighbour(p, x, y, z, VEL[i][0], VEL[i][1], VEL[i][2]);
                int ty = type_of(p, nb);
                if (ty == ORC_FLUID) {
                    B[(int64_t)i * n + nb] = fs[i];
                } else {
                    int r = inverse(q, i);
                    B[(int64_t)r * n + v] = bc_value(p, ty, fs[i], r, inlet_velocity(p, rank, nb), uc);
                }
            }
        }
        double *tmp = A; A = B; B = tmp;
    }
    if (A != f) {
        memcpy(f, A, sizeof(double) * (size_t)(q * n));
        B = A;
    }
    free(B);
    free(rank);
    return 0;
}

/* rho, u (Guo-corrected) per voxel; non-fluid voxels get rho = 0, u = 0. */
void orc_dense_macroscopic(const orc_problem *p, const double *f, double *rho, double *u) {
    int64_t n = nvox(p);
    for (int64_t v = 0; v < n; ++v) {
        if (p->flags[v] != ORC_FLUID) {
            rho[v] = 0.0;
            u[3 * v] = u[3 * v + 1] = u[3 * v + 2] = 0.0;
            continue;
        }
        double fl[27];
        for (int i = 0; i < p->q; ++i) fl[i] = f[(int64_t)i * n + v];
        orc_moments(p->q, fl, p->force, &rho[v], &u[3 * v]);
    }
}

/* rho, u (Guo-corrected) of every cell of a PDF-list (Q x S, slot i*S + k). */
void orc_sparse_macroscopic(const orc_problem *p, const double *f, int64_t nf, int64_t S, double *rho, double *u) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nf; ++k) {
        double fl[27];
        for (int i = 0; i < p->q; ++i) fl[i] = f[(int64_t)i * S + k];
        orc_moments(p->q, fl, p->force, &rho[k], &u[3 * k]);
    }
}

/* ------------------------------------------------------- sparse indexing */

/* Compacted fluid-cell order (Sec. 3.1): fluid voxels numbered in
 * ascending linear voxel id (lexicographic, x fastest).  cell_id[v] = k or
 * -1; cell_voxel[k] = v.  Returns N_F. */
/* Compacted fluid-cell order (Sec. 3.1).  order 0: voxels lexicographic,
 * x fastest.  order 1 ("brick-8"): the box is cut into 8x8x8 bricks taken in
 * lexicographic brick order, and the voxels of each brick lexicographically
 * (bricks at the high faces may be partial).  Fluid voxels are numbered in
 * that visiting order. */
static void visit(const orc_problem *p, int64_t v, int64_t *k, int32_t *cell_id, int32_t *cell_voxel) {
    if (p->flags[v] == ORC_FLUID) {
        cell_id[v] = (int32_t)*k;
        cell_voxel[*k] = (int32_t)v;
        ++*k;
    } else {
        cell_id[v] = -1;
    }
}

/* A brick is "full" when it lies wholly inside the box (8x8x8 voxels) and
 * every voxel of it is fluid. */
static int brick_full(const orc_problem *p, int bx, int by, int bz) {
    if (bx + 8 > p->nx || by + 8 > p->ny || bz + 8 > p->nz) return 0;
    for (int z = bz; z < bz + 8; ++z)
        for (int y = by; y < by + 8; ++y)
            for (int x = bx; x < bx + 8; ++x)
                if (p->flags[x + (int64_t)p->nx * (y + (int64_t)p->ny * z)] != ORC_FLUID) return 0;
    return 1;
}

/* order 2 ("hybrid"): first the full bricks, in lexicographic brick order
 * and lexicographic inside each; then every other fluid voxel in the brick-8
 * order (the full bricks skipped).  The cells of a full brick are 512
 * consecutive cells, whose neighbours inside the brick follow from the cell
 * number alone (the dense part of a hybrid sparse/dense layout, Sec. 4.1). */
int64_t orc_compact(const orc_problem *p, int32_t *cell_id, int32_t *cell_voxel) {
    int64_t n = nvox(p), k = 0;
    if (p->order == 0) {
        for (int64_t v = 0; v < n; ++v) visit(p, v, &k, cell_id, cell_voxel);
        return k;
    }
    for (int pass = (p->order == 2 ? 0 : 1); pass < 2; ++pass)
        for (int bz = 0; bz < p->nz; bz += 8)
            for (int by = 0; by < p->ny; by += 8)
                for (int bx = 0; bx < p->nx; bx += 8) {
                    if (p->order == 2 && brick_full(p, bx, by, bz) != (pass == 0)) continue;
                    for (int z = bz; z < bz + 8 && z < p->nz; ++z)
                        for (int y = by; y < by + 8 && y < p->ny; ++y)
                            for (int x = bx; x < bx + 8 && x < p->nx; ++x)
                                visit(p, x + (int64_t)p->nx * (y + (int64_t)p->ny * z), &k, cell_id, cell_voxel);
                }
    return k;
}

#define ORC_PAD INT32_MIN

/* Pull index-list (Sec. 3.1, Sec. 3.1.1).  Row r = i-1 for i = 1..Q-1,
 * column k, stride S (>= N_F):
 *   fluid neighbour x_k - c_i      -> i*S + cell_id(neighbour)
 *   wall (or outside, non-periodic)-> inverse(i)*S + k      (same cell, inverse dir)
 *   inlet / outlet voxel           -> -(b+1), b = running link number in
 *                                     (k, i) order
 *   padding columns k >= N_F       -> INT32_MIN
 * Link table (n_bc entries, up to max_bc written): cell, direction,
 * boundary type, and the inlet velocity of the boundary voxel.
 * Returns the number of boundary links. */
int64_t orc_pull_list(const orc_problem *p, const int32_t *cell_id, const int32_t *cell_voxel,
                      int64_t nf, int64_t S, int32_t *P, int32_t *bc_cell, int32_t *bc_dir,
                      int32_t *bc_type, double *bc_u, int64_t max_bc) {
    int q = p->q;
    int64_t nb_links = 0;
    int64_t *rank = inlet_rank(p);
    for (int i = 1; i < q; ++i)
        for (int64_t k = nf; k < S; ++k) P[(int64_t)(i - 1) * S + k] = ORC_PAD;
    for (int64_t k = 0; k < nf; ++k) {
        int64_t v = cell_voxel[k];
        int x = (int)(v % p->nx), y = (int)((v / p->nx) % p->ny), z = (int)(v / ((int64_t)p->nx * p->ny));
        for (int i = 1; i < q; ++i) {
            int64_t nb = neighbour(p, x, y, z, -VEL[i][0], -VEL[i][1], -VEL[i][2]);
            int ty = type_of(p, nb);
            int32_t val;
            if (ty == ORC_FLUID) {
                val = (int32_t)((int64_t)i * S + cell_id[nb]);
            } else if (ty == ORC_WALL) {
                val = (int32_t)((int64_t)inverse(q, i) * S + k);
            } else {
                if (nb_links < max_bc) {
                    bc_cell[nb_links] = (int32_t)k;
                    bc_dir[nb_links] = i;
                    bc_type[nb_links] = ty;
                    const double *uw = inlet_velocity(p, rank, nb);
                    for (int a = 0; a < 3; ++a) bc_u[3 * nb_links + a] = uw[a];
                }
                val = (int32_t)(-(nb_links + 1));
                ++nb_links;
            }
            P[(int64_t)(i - 1) * S + k] = val;
        }
    }
    free(rank);
    return nb_links;
}

/* ---------------------------------------------------- sparse stepping */

/* Two-grid PULL stepping over the PDF-list (Q x S, slot i*S + k):
 * collide every cell into C (keeping each cell's velocity), then
 * f_i(k) <- C[P(i,k)] for fluid/wall links and the boundary value of
 * C[inverse(i)*S + k] for inlet/outlet links.  Uses the same per-cell
 * arithmetic as orc_dense_run, so the two agree bit for bit. */
int orc_sparse_run(const orc_problem *p, const int32_t *P, int64_t nf, int64_t S,
                   const int32_t *bc_type, const double *bc_u, double *f, int steps) {
    int q = p->q;
    double *C = (double *)malloc(sizeof(double) * (size_t)(q * S > 0 ? q * S : 1));
    double *U = (double *)malloc(sizeof(double) * (size_t)(3 * nf > 0 ? 3 * nf : 1));
    if (!C || !U) {
        free(C);
        free(U);
        return -1;
    }
    for (int t = 0; t < steps; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k) {
            double fl[27], fs[27], rho;
            for (int i = 0; i < q; ++i) fl[i] = f[(int64_t)i * S + k];
            orc_moments(q, fl, p->force, &rho, &U[3 * k]);
            orc_collide(p, fl, fs);
            for (int i = 0; i < q; ++i) C[(int64_t)i * S + k] = fs[i];
        }
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nf; ++k) {
            f[k] = C[k];
            for (int i = 1; i < q; ++i) {
                int32_t e = P[(int64_t)(i - 1) * S + k];
                if (e >= 0) {
                    f[(int64_t)i * S + k] = C[e];
                } else {
                    int64_t b = -(int64_t)e - 1;
                    int r = inverse(q, i);
                    f[(int64_t)i * S + k] =
                        bc_value(p, bc_type[b], C[(int64_t)r * S + k], i, bc_u + 3 * b, &U[3 * k]);
                }
            }
        }
    }
    free(C);
    free(U);
    return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
