"""FP64 CPU oracle for the sparse AA lattice Boltzmann path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product library (``paper_2408_06880_gb300``) never imports, links or runs it,
and it imports nothing from the product.  The only code both sides share is the
seeded input generator package ``geometry`` (no LBM arithmetic there).

Contents (each function cites the passage it follows):

* ``oracle.c`` (plain C, FP64, compiled here with gcc): stencils, Eq. 1
  moments, Eq. 6 equilibrium, Eq. 5 SRT / textbook TRT / D3Q19 MRT (the
  orthogonal moment basis of d'Humieres et al. 2002) / D3Q27 central-moment
  and cumulant (Geier et al. 2015) collisions with a Guo force (Sec. 4 lists
  these operators, Sec. 5.1 benchmarks them), a dense direct-addressing
  two-grid PUSH stepper (Sec. 2-3), the
  compacted cell order and the pull index-list (Sec. 3.1, 3.1.1) and a sparse
  two-grid PULL stepper on that list.
* this module: ctypes marshalling, the TRT rate from the magic parameter, the
  permeability definition, and the paper's memory-access and memory-footprint
  models (Tables 1 and 2 of Sec. 5.1, Eq. 9 of Sec. 4 and Eq. 11 of Sec. 5.1).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, brute force on tiny inputs, the paper's printed
table values); the inlet/outlet boundary maps are pinned only by Couette
(closed form) and a plug-flow flux invariant.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

SRT, TRT, MRT, CM, CUMULANT = 0, 1, 2, 3, 4
FLUID, WALL, INLET, OUTLET = 0, 1, 2, 3
PAD = np.iinfo(np.int32).min


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA
    contraction so x86 and Arm give identical bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("flags", C.c_void_p), ("periodic", C.c_uint32), ("q", C.c_int32),
                ("op", C.c_int32), ("omega_plus", C.c_double), ("omega_minus", C.c_double),
                ("force", C.c_double * 3), ("inlet_u", C.c_void_p), ("rho_out", C.c_double),
                ("mrt_s", C.c_double * 19), ("order", C.c_int32), ("cm_bulk", C.c_double),
                ("cm_high", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER(_Problem)
            vp, i64 = C.c_void_p, C.c_int64
            L.orc_stencil.argtypes = [C.c_int, vp, vp, vp]
            L.orc_equilibrium.argtypes = [C.c_int, C.c_double, vp, vp]
            L.orc_guo_source.argtypes = [C.c_int, vp, vp, vp]
            L.orc_moments.argtypes = [C.c_int, vp, vp, vp, vp]
            L.orc_collide.argtypes = [P, vp, vp]
            L.orc_mrt_matrix.argtypes = [vp]
            L.orc_central_moments.argtypes = [vp, vp, vp]
            L.orc_from_central.argtypes = [vp, vp, vp]
            L.orc_cumulants.argtypes = [P, vp, vp]
            L.orc_dense_init.argtypes = [P, vp, vp, vp]
            L.orc_dense_run.argtypes = [P, vp, C.c_int]
            L.orc_dense_macroscopic.argtypes = [P, vp, vp, vp]
            L.orc_compact.argtypes = [P, vp, vp]
            L.orc_compact.restype = i64
            L.orc_pull_list.argtypes = [P, vp, vp, i64, i64, vp, vp, vp, vp, vp, i64]
            L.orc_pull_list.restype = i64
            L.orc_sparse_run.argtypes = [P, vp, i64, i64, vp, vp, vp, C.c_int]
            L.orc_sparse_macroscopic.argtypes = [P, vp, i64, i64, vp, vp]
            L.orc_max_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ----------------------------------------------------------------- problem

def trt_omega_minus(omega_plus: float, magic: float) -> float:
    """TRT odd relaxation rate from the magic parameter
    Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) (textbook TRT, named in Sec. 4)."""
    return 1.0 / (magic / (1.0 / omega_plus - 0.5) + 0.5)


def mrt_default_rates(omega: float) -> tuple:
    """Per-moment MRT rates of d'Humieres et al. (2002) for the D3Q19 basis
    order (rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy,
    pyz, pxz, mx, my, mz): conserved moments 0, s_e = 1.19, s_eps = s_pi =
    1.4, s_q = 1.2, s_m = 1.98, and omega (Eq. 7) on the stress moments."""
    w = float(omega)
    return (0.0, 1.19, 1.4, 0.0, 1.2, 0.0, 1.2, 0.0, 1.2, w, 1.4, w, 1.4, w, w, w, 1.98, 1.98, 1.98)


def mrt_matrix() -> np.ndarray:
    """The oracle's D3Q19 MRT moment matrix M[a, i] (rows: the basis of
    d'Humieres et al. 2002, columns: the velocity table)."""
    M = np.zeros((19, 19))
    lib().orc_mrt_matrix(_ptr(M))
    return M


@dataclass
class Problem:
    """A voxel geometry plus the method's parameters (Sec. 2: stencil,
    collision operator, relaxation rate(s), body force)."""

    flags: np.ndarray                 # uint8 (nz, ny, nx)
    periodic: int = 7
    q: int = 19
    op: int = SRT
    omega_plus: float = 1.0 / 0.8
    magic: float = 3.0 / 16.0
    force: tuple = (0.0, 0.0, 0.0)
    inlet_u: np.ndarray | None = None
    rho_out: float = 1.0
    mrt_rates: tuple | None = None    # MRT: 19 per-moment rates (default mrt_default_rates)
    cm_bulk: float = 1.0              # CM / CUMULANT (D3Q27): rate of the trace of the second moments
    cm_high: float = 1.0              # CM / CUMULANT: rate of the moments (cumulants) of orders 3..6
    order: int = 0                    # cell order: 0 lexicographic, 1 brick-8, 2 full bricks first

    @classmethod
    def from_geometry(cls, g, **kw):
        return cls(flags=g.flags, periodic=g.periodic, inlet_u=g.inlet_u, rho_out=g.rho_out, **kw)

    @property
    def shape(self):
        nz, ny, nx = self.flags.shape
        return nx, ny, nz

    @property
    def n(self) -> int:
        return int(self.flags.size)

    @property
    def omega_minus(self) -> float:
        if self.op == SRT:
            return self.omega_plus
        return trt_omega_minus(self.omega_plus, self.magic)

    @property
    def nu(self) -> float:
        """Eq. 7: nu = c_s^2 (1/omega - 1/2)."""
        return (1.0 / self.omega_plus - 0.5) / 3.0

    def _c(self):
        self._flags_c = np.ascontiguousarray(self.flags, dtype=np.uint8)
        self._inlet_c = (None if self.inlet_u is None
                         else np.ascontiguousarray(self.inlet_u, dtype=np.float64).reshape(-1))
        nx, ny, nz = self.shape
        if self.op == MRT and self.q != 19:
            raise ValueError("the MRT operator is defined for D3Q19")
        if self.op in (CM, CUMULANT) and self.q != 27:
            raise ValueError("the central-moment and cumulant operators are defined for D3Q27")
        rates = self.mrt_rates if self.mrt_rates is not None else mrt_default_rates(self.omega_plus)
        s = _Problem(nx, ny, nz, _ptr(self._flags_c), self.periodic, self.q, self.op,
                     self.omega_plus, self.omega_minus, (C.c_double * 3)(*self.force),
                     _ptr(self._inlet_c), self.rho_out, (C.c_double * 19)(*rates), self.order,
                     self.cm_bulk, self.cm_high)
        self._cs = s
        return C.byref(s)


# ----------------------------------------------------------------- stencil

def stencil(q: int):
    """Velocity set (c[Q,3], w[Q], inverse[Q]) of D3Q19 / D3Q27."""
    c = np.zeros((q, 3), np.int32)
    w = np.zeros(q)
    inv = np.zeros(q, np.int32)
    if lib().orc_stencil(q, _ptr(c), _ptr(w), _ptr(inv)) != 0:
        raise ValueError("q must be 19 or 27")
    return c, w, inv


def equilibrium(q: int, rho: float, u) -> np.ndarray:
    """Eq. 6 second-order equilibrium, c_s^2 = 1/3."""
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(q)
    lib().orc_equilibrium(q, rho, _ptr(u), _ptr(out))
    return out


def guo_source(q: int, u, F) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    F = np.ascontiguousarray(F, np.float64)
    out = np.zeros(q)
    lib().orc_guo_source(q, _ptr(u), _ptr(F), _ptr(out))
    return out


def central_moments(f, u) -> np.ndarray:
    """D3Q27 central moments about u: [a + 3b + 9c] = sum f (cx-ux)^a (cy-uy)^b (cz-uz)^c."""
    f = np.ascontiguousarray(f, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(27)
    lib().orc_central_moments(_ptr(f), _ptr(u), _ptr(out))
    return out


def from_central(kap, u) -> np.ndarray:
    """The D3Q27 populations with the given central moments about u."""
    kap = np.ascontiguousarray(kap, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    out = np.zeros(27)
    lib().orc_from_central(_ptr(kap), _ptr(u), _ptr(out))
    return out


def cumulants(p: Problem, f) -> np.ndarray:
    """Normalised cumulants (orders >= 2, moment indexing) of one D3Q27 cell
    about its Guo velocity; orders 0 and 1 as 0."""
    f = np.ascontiguousarray(f, np.float64)
    out = np.zeros(27)
    lib().orc_cumulants(p._c(), _ptr(f), _ptr(out))
    return out


def collide(p: Problem, f) -> np.ndarray:
    """One cell's post-collision PDFs (Eq. 3)."""
    f = np.ascontiguousarray(f, np.float64)
    out = np.zeros(p.q)
    lib().orc_collide(p._c(), _ptr(f), _ptr(out))
    return out


# ------------------------------------------------------------------ dense

def dense_init(p: Problem, rho=None, u=None) -> np.ndarray:
    """f = f^eq(rho, u) on fluid voxels (rest state when rho, u are None)."""
    f = np.zeros((p.q, p.n))
    r = None if rho is None else np.ascontiguousarray(rho, np.float64)
    uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1)
    lib().orc_dense_init(p._c(), _ptr(r), _ptr(uu), _ptr(f))
    return f


def dense_run(p: Problem, f: np.ndarray, steps: int) -> np.ndarray:
    """`steps` two-grid push steps (Eqs. 3-4) in place on a copy of f."""
    f = np.ascontiguousarray(f, np.float64).copy()
    if lib().orc_dense_run(p._c(), _ptr(f), int(steps)) != 0:
        raise MemoryError("oracle dense_run")
    return f


def dense_macroscopic(p: Problem, f: np.ndarray):
    """(rho[N], u[N,3]) with the Guo half-force velocity; zeros off-fluid."""
    rho = np.zeros(p.n)
    u = np.zeros((p.n, 3))
    lib().orc_dense_macroscopic(p._c(), _ptr(np.ascontiguousarray(f)), _ptr(rho), _ptr(u))
    return rho, u


# ----------------------------------------------------------------- sparse

def stride_of(nf: int) -> int:
    """PDF-list stride: N_F rounded up to a multiple of 128."""
    return (nf + 127) // 128 * 128


def compact(p: Problem):
    """Compacted fluid-cell order (Sec. 3.1) by `p.order`: lexicographic,
    brick-8, or full 8^3 bricks first then the rest in brick-8 order:
    (cell_id[N], cell_voxel[N_F])."""
    cid = np.zeros(p.n, np.int32)
    cvx = np.zeros(max(p.n, 1), np.int32)
    nf = lib().orc_compact(p._c(), _ptr(cid), _ptr(cvx))
    return cid, cvx[:nf].copy()


@dataclass
class Lists:
    cell_id: np.ndarray
    cell_voxel: np.ndarray
    n_fluid: int
    stride: int
    P: np.ndarray            # int32 (Q-1, S)
    bc_cell: np.ndarray
    bc_dir: np.ndarray
    bc_type: np.ndarray
    bc_u: np.ndarray         # (n_bc, 3)


def pull_list(p: Problem) -> Lists:
    """Pull index-list with no-slip and periodic folded in and inlet/outlet
    links as negative link ids (Sec. 3.1, 3.1.1)."""
    cid, cvx = compact(p)
    nf = int(cvx.size)
    S = stride_of(nf)
    P = np.zeros((p.q - 1, S), np.int32)
    # count links first with max_bc = 0, then fill
    L = lib()
    nb = L.orc_pull_list(p._c(), _ptr(cid), _ptr(cvx), nf, S, _ptr(P), None, None, None, None, 0)
    bc_cell = np.zeros(max(nb, 1), np.int32)
    bc_dir = np.zeros(max(nb, 1), np.int32)
    bc_type = np.zeros(max(nb, 1), np.int32)
    bc_u = np.zeros((max(nb, 1), 3))
    L.orc_pull_list(p._c(), _ptr(cid), _ptr(cvx), nf, S, _ptr(P), _ptr(bc_cell), _ptr(bc_dir),
                    _ptr(bc_type), _ptr(bc_u), nb)
    return Lists(cid, cvx, nf, S, P, bc_cell[:nb], bc_dir[:nb], bc_type[:nb], bc_u[:nb])


def sparse_from_dense(lists: Lists, f_dense: np.ndarray) -> np.ndarray:
    """Gather the fluid columns of a dense Q x N field into a Q x S list."""
    q = f_dense.shape[0]
    out = np.zeros((q, lists.stride))
    out[:, :lists.n_fluid] = f_dense[:, lists.cell_voxel]
    return out


def sparse_run(p: Problem, lists: Lists, f: np.ndarray, steps: int) -> np.ndarray:
    """`steps` two-grid pull steps over the PDF-list (Sec. 3.1)."""
    f = np.ascontiguousarray(f, np.float64).copy()
    bt = np.ascontiguousarray(lists.bc_type if lists.bc_type.size else np.zeros(1, np.int32))
    bu = np.ascontiguousarray(lists.bc_u if lists.bc_u.size else np.zeros((1, 3)))
    if lib().orc_sparse_run(p._c(), _ptr(lists.P), lists.n_fluid, lists.stride, _ptr(bt),
                            _ptr(bu), _ptr(f), int(steps)) != 0:
        raise MemoryError("oracle sparse_run")
    return f


def sparse_rest(p: Problem, lists: Lists) -> np.ndarray:
    """The rest state on a PDF-list: f_i = w_i (the equilibrium at rho = 1,
    u = 0) in every fluid column, zero padding."""
    _, w, _ = stencil(p.q)
    f = np.zeros((p.q, lists.stride))
    f[:, :lists.n_fluid] = w[:, None]
    return f


def sparse_macroscopic(p: Problem, lists: Lists, f: np.ndarray):
    """(rho[N_F], u[N_F,3]) of a PDF-list, Guo half-force velocity (Eq. 1)."""
    nf = lists.n_fluid
    rho = np.zeros(max(nf, 1))
    u = np.zeros((max(nf, 1), 3))
    lib().orc_sparse_macroscopic(p._c(), _ptr(np.ascontiguousarray(f)), nf, lists.stride, _ptr(rho), _ptr(u))
    return rho[:nf], u[:nf]


# ------------------------------------------------------- derived quantities

def reductions(p: Problem, f: np.ndarray):
    """The five FP64 domain sums of the macroscopic state, in the order
    (sum(rho-1), sum rho*u_x, sum rho*u_y, sum rho*u_z, sum u_x) over fluid
    voxels, with the Guo half-force velocity."""
    rho, u = dense_macroscopic(p, f)
    m = p.flags.reshape(-1) == FLUID
    r, uu = rho[m], u[m]
    return np.array([np.sum(r - 1.0), np.sum(r * uu[:, 0]), np.sum(r * uu[:, 1]),
                     np.sum(r * uu[:, 2]), np.sum(uu[:, 0])])


def permeability(p: Problem, sum_ux: float) -> float:
    """Darcy permeability in lattice units^2: k = nu * U_D / F_x with the
    superficial velocity U_D = sum_fluid u_x / N (rho0 = 1)."""
    return p.nu * (sum_ux / p.n) / p.force[0]


def max_threads() -> int:
    return int(lib().orc_max_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ------------------------------------------- paper's byte and memory models

def access_bytes(q: int, b_pdf: int, b_idx: int, pattern: str, data: str, arch: str) -> float:
    """Memory accesses per cell update (Tables 1 and 2, Sec. 5.1).

    pattern 'pull' or 'aa'; data 'dense' or 'sparse'; arch 'cpu' adds the
    write-allocate of the pull pattern's second field."""
    if pattern == "pull":
        pdf = (3 if arch == "cpu" else 2) * q * b_pdf
        idx = (q - 1) * b_idx
    elif pattern == "aa":
        pdf = 2 * q * b_pdf
        idx = (q - 1) / 2 * b_idx
    else:
        raise ValueError(pattern)
    return pdf + (idx if data == "sparse" else 0)


def memory_bytes_per_cell(q: int, b_pdf: int, b_idx: int, layout: str, porosity: float) -> float:
    """Memory per lattice cell (Eq. 9, Sec. 4, and its AA variant Eq. 11):
    sparse two-grid N(2QB + (Q-1)B_idx + 5B)phi, dense N(2QB + 5B),
    sparse AA N(QB + (Q-1)B_idx + 5B)phi; 5B covers velocity, density and
    flag fields."""
    if layout == "sparse":
        return (2 * q * b_pdf + (q - 1) * b_idx + 5 * b_pdf) * porosity
    if layout == "dense":
        return 2 * q * b_pdf + 5 * b_pdf
    if layout == "sparse_aa":
        return (q * b_pdf + (q - 1) * b_idx + 5 * b_pdf) * porosity
    raise ValueError(layout)
