"""Python face of the C ABI: one `Domain` per sparse (or dense comparator)
lattice Boltzmann domain.  Argument marshalling only -- every step of the
method runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _capi as A


def validate_pull_list(P: np.ndarray, n_fluid: int, n_links: int) -> None:
    """Host-side check of a canonical pull index-list (Sec. 3.1, 3.1.1), as
    exported by `Domain.export_lists`: rows i-1 = directions i = 1..Q-1,
    stride S = P.shape[1].  Column k < n_fluid holds i*S + n (fluid neighbour
    n < n_fluid), inverse(i)*S + k (wall: the cell's own inverse slot) or
    -(b+1) with b < n_links (inlet/outlet link); padding columns hold
    INT32_MIN.  Raises ValueError naming the first bad entry."""
    P = np.asarray(P, np.int64)
    q = P.shape[0] + 1
    S = P.shape[1]
    if S < n_fluid or S % 128:
        raise ValueError(f"stride {S} does not hold {n_fluid} cells in multiples of 128")
    k = np.arange(n_fluid)
    pad = np.iinfo(np.int32).min
    for r in range(q - 1):
        i = r + 1
        ib = i + 1 if i % 2 else i - 1                      # inverse pairs (i, i+1), i odd
        e = P[r, :n_fluid]
        fluid = (e >= i * S) & (e < i * S + n_fluid)
        wall = e == ib * S + k
        link = (e < 0) & (e >= -n_links)
        bad = ~(fluid | wall | link)
        if bad.any():
            j = int(np.argmax(bad))
            raise ValueError(f"direction {i}, cell {j}: entry {int(e[j])} is no fluid, wall or link slot")
        if np.any(P[r, n_fluid:] != pad):
            raise ValueError(f"direction {i}: a padding column is not INT32_MIN")


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator.

    The library calls `alloc`/`free` through C function pointers; each
    allocation is a uint8 CUDA tensor kept alive here until freed."""

    def __init__(self, device=None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.live: dict[int, object] = {}
        self._alloc = A.ALLOC_FN(self._do_alloc)
        self._free = A.FREE_FN(self._do_free)
        self.struct = A.Allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, _ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
        except Exception:       # out of memory -> NULL, the library reports ENOMEM
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _do_free(self, ptr, _ctx):
        self.live.pop(int(ptr), None)

    @property
    def bytes(self) -> int:
        return sum(t.numel() for t in self.live.values())


def auto_scale_exp(u_max: float, drho_max: float = 0.0, target: float = 4096.0) -> int:
    """Power-of-two storage exponent for FP16/BF16 so that the largest
    shifted population (about u_max/6 + drho_max/3) maps near `target`."""
    gmax = max(u_max / 6.0 + drho_max / 3.0, 1e-30)
    return int(max(-40, min(40, math.floor(math.log2(target / gmax)))))


class Domain:
    """A compacted sparse (or dense comparator) LBM domain on the GPU."""

    def __init__(self, flags: np.ndarray, *, periodic: int = 7, q: int = 19, op: int = A.SRT,
                 omega: float = 1.25, trt_magic: float = 3.0 / 16.0, force=(0.0, 0.0, 0.0),
                 inlet_u: np.ndarray | None = None, rho_out: float = 1.0, storage: int = A.FP32,
                 scale_exp: int = 0, layout: int = A.SPARSE, stream=None, allocator="torch",
                 cell_order: int = A.ORDER_LEX):
        L = A.lib()
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        if flags.ndim != 3:
            raise ValueError("flags must be a (nz, ny, nx) array")
        nz, ny, nx = flags.shape
        self._flags = flags
        self._inlet = None if inlet_u is None else np.ascontiguousarray(inlet_u, dtype=np.float32).reshape(-1, 3)
        d = A.Desc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.flags = flags.ctypes.data
        d.periodic = periodic
        d.q, d.op = q, op
        d.omega_plus, d.trt_magic = omega, trt_magic
        d.force = (C.c_double * 3)(*force)
        d.inlet_u = None if self._inlet is None else self._inlet.ctypes.data
        d.n_inlet_u = 0 if self._inlet is None else self._inlet.shape[0]
        d.rho_out = rho_out
        d.storage, d.scale_exp, d.layout, d.order = storage, scale_exp, layout, cell_order
        self.desc = d
        self.params = dict(q=q, op=op, omega=omega, trt_magic=trt_magic, force=tuple(force),
                           storage=storage, scale_exp=scale_exp, layout=layout, periodic=periodic,
                           cell_order=cell_order)
        self.shape = (nx, ny, nz)
        self._alloc = TorchAllocator() if allocator == "torch" else None
        self._stream = stream
        sp = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        h = C.c_void_p()
        A.check(L.sparse_lbm_create(C.byref(d), None if self._alloc is None else C.byref(self._alloc.struct),
                                    sp or None, C.byref(h)))
        self.h = h

    # ------------------------------------------------------------- basics
    def close(self):
        if getattr(self, "h", None):
            A.lib().sparse_lbm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def info(self) -> dict:
        i = A.Info()
        A.check(A.lib().sparse_lbm_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in A.Info._fields_ if f != "pad"}

    @property
    def n_fluid(self) -> int:
        return self.info["n_fluid"]

    @property
    def step_count(self) -> int:
        return self.info["step"]

    @property
    def nu(self) -> float:
        return (1.0 / self.params["omega"] - 0.5) / 3.0

    # -------------------------------------------------------------- stepping
    def step(self, n: int = 1, graph: bool = False):
        fn = A.lib().sparse_lbm_step_graph if graph else A.lib().sparse_lbm_step
        A.check(fn(self.h, int(n)))

    def set_launch(self, parity: int, threads: int, cells: int, variant: int = 0):
        """variant 0: `cells` consecutive cells per thread; variant 1: persistent
        CTAs of `threads`-cell tiles with `cells` bulk-staged tiles in flight;
        odd step: variant 2 L2 index prefetch, 3 re-read slots, 4 16-bit codes."""
        A.check(A.lib().sparse_lbm_set_launch(self.h, parity, threads, cells, variant))

    def set_cm_rates(self, bulk: float = 1.0, higher: float = 1.0):
        """Central-moment and cumulant domains: the rate of the trace of the
        second-order central moments and of the moments of order 3..6
        (cumulant domains: higher == 1)."""
        A.check(A.lib().sparse_lbm_set_cm_rates(self.h, float(bulk), float(higher)))

    def set_mrt_rates(self, rates):
        """MRT domains: the 19 per-moment relaxation rates (basis order rho, e,
        eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx,
        my, mz; conserved entries ignored)."""
        r = np.ascontiguousarray(rates, np.float64)
        if r.shape != (19,):
            raise ValueError("19 rates")
        A.check(A.lib().sparse_lbm_set_mrt_rates(self.h, r.ctypes.data))

    def set_checked(self, on: bool):
        A.check(A.lib().sparse_lbm_set_checked(self.h, int(bool(on))))

    def device_error(self) -> int:
        code = C.c_int32()
        st = A.lib().sparse_lbm_device_error(self.h, C.byref(code))
        if st not in (A.OK, A.EDEVICE):
            A.check(st)
        return code.value

    # ------------------------------------------------------------ outputs
    def macroscopic(self, order: int = A.ORDER_CELLS):
        """(rho[n], u[3, n]) as host numpy float32 arrays."""
        n = self.info["n_voxels"] if order == A.ORDER_VOXELS or self.params["layout"] == A.DENSE \
            else self.n_fluid
        rho = np.zeros(n, np.float32)
        u = np.zeros((3, n), np.float32)
        A.check(A.lib().sparse_lbm_macroscopic(self.h, rho.ctypes.data, u.ctypes.data, order, A.MEM_HOST))
        return rho, u

    def macroscopic_device(self, rho, u, order: int = A.ORDER_CELLS):
        """Fill CUDA tensors rho[n], u[3, n] (float32) asynchronously."""
        A.check(A.lib().sparse_lbm_macroscopic(self.h, rho.data_ptr() if rho is not None else None,
                                               u.data_ptr() if u is not None else None, order, A.MEM_DEVICE))

    def reduce(self) -> np.ndarray:
        """FP64 sums: [sum(rho-1), sum rho u_x, sum rho u_y, sum rho u_z, sum u_x]."""
        out = np.zeros(5)
        A.check(A.lib().sparse_lbm_reduce(self.h, out.ctypes.data, A.MEM_HOST))
        return out

    def reduce_device(self, out):
        A.check(A.lib().sparse_lbm_reduce(self.h, out.data_ptr(), A.MEM_DEVICE))

    def reduce_ext(self, check: bool = True) -> np.ndarray:
        """The five FP64 sums plus max |f_i - w_i| (unscaled) and max |u|.
        check=False returns the values even when one is not finite or the
        largest speed exceeds 0.3 (the library then reports EDIVERGED)."""
        out = np.zeros(7)
        st = A.lib().sparse_lbm_reduce_ext(self.h, out.ctypes.data, A.MEM_HOST)
        if st != A.OK and (check or st != A.EDIVERGED):
            A.check(st)
        return out

    def reduce_ext_device(self, out):
        A.check(A.lib().sparse_lbm_reduce_ext(self.h, out.data_ptr(), A.MEM_DEVICE))

    def set_storage(self, storage: int, scale_exp: int = 0):
        """Convert the stored populations to another storage format or
        power-of-two scale in place (exact for FP16/BF16 -> FP32 and for
        rescales; FP32 -> FP16/BF16 rounds to nearest).  The domain must not
        be a pool member."""
        A.check(A.lib().sparse_lbm_set_storage(self.h, int(storage), int(scale_exp)))
        inf = self.info
        self.params["storage"], self.params["scale_exp"] = inf["storage"], inf["scale_exp"]

    def permeability(self, sums: np.ndarray | None = None) -> float:
        """Darcy permeability nu * U_D / F_x, U_D = sum u_x / N (lattice units^2)."""
        s = self.reduce() if sums is None else sums
        return self.nu * (s[4] / self.info["n_voxels"]) / self.params["force"][0]

    def init_equilibrium(self, rho=None, u=None, order: int = A.ORDER_VOXELS):
        r = None if rho is None else np.ascontiguousarray(rho, np.float32)
        uu = None if u is None else np.ascontiguousarray(u, np.float32)
        A.check(A.lib().sparse_lbm_init_equilibrium(self.h, None if r is None else r.ctypes.data,
                                                    None if uu is None else uu.ctypes.data, order,
                                                    A.MEM_HOST))

    def export_lists(self) -> dict:
        inf = self.info
        nf, S, q, nl = inf["n_fluid"], inf["stride"], inf["q"], inf["n_bc_links"]
        cv = np.zeros(max(nf, 1), np.int32)
        P = np.zeros((q - 1, max(S, 1)), np.int32)
        lc, ld, lt = (np.zeros(max(nl, 1), np.int32) for _ in range(3))
        A.check(A.lib().sparse_lbm_export_lists(self.h, cv.ctypes.data, P.ctypes.data, lc.ctypes.data,
                                                ld.ctypes.data, lt.ctypes.data))
        return dict(cell_voxel=cv[:nf], P=P[:, :S], link_cell=lc[:nl], link_dir=ld[:nl], link_type=lt[:nl],
                    n_fluid=nf, stride=S)

    def validate_lists(self) -> None:
        """Check every entry of the device's index-list on the host
        (`validate_pull_list`)."""
        L = self.export_lists()
        validate_pull_list(L["P"], L["n_fluid"], int(L["link_cell"].size))

    def export_codes(self) -> tuple[np.ndarray, np.ndarray]:
        """The odd step's 16-bit link codes ((Q-1) x S uint16) and their
        column bases ((S/128) x (Q-1) int32)."""
        inf = self.info
        S, q = inf["stride"], inf["q"]
        codes = np.zeros((q - 1, max(S, 1)), np.uint16)
        bases = np.zeros((max(S // 128, 1), q - 1), np.int32)
        A.check(A.lib().sparse_lbm_export_codes(self.h, codes.ctypes.data, bases.ctypes.data))
        return codes[:, :S], bases[:S // 128]

    def get_state(self):
        nb = C.c_int64()
        A.check(A.lib().sparse_lbm_state_bytes(self.h, C.byref(nb)))
        buf = np.zeros(nb.value, np.uint8)
        step = C.c_int64()
        A.check(A.lib().sparse_lbm_get_state(self.h, buf.ctypes.data, C.byref(step)))
        return buf, step.value

    def set_state(self, buf: np.ndarray, step: int):
        buf = np.ascontiguousarray(buf, np.uint8)
        A.check(A.lib().sparse_lbm_set_state(self.h, buf.ctypes.data, int(step)))

    def memory_bytes(self) -> int:
        return self.info["device_bytes"]
