"""Batched stepping: many domains advanced by one persistent kernel per time
step (C ABI slbm_pool_*).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _capi as A


class Pool:
    """A set of sparse domains (same stencil and storage) stepped together.

    The pool does not own its members.  While a domain is a member, step it
    through the pool only; `reduce()` synchronises the pool's stream, after
    which member handles may be read directly."""

    def __init__(self, q: int = 19, storage: int = A.FP32, capacity: int = 64, stream=None):
        self.q, self.storage, self.capacity = q, storage, capacity
        self._stream = stream
        sp = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        h = C.c_void_p()
        A.check(A.lib().slbm_pool_create(q, storage, capacity, sp or None, C.byref(h)))
        self.h = h
        self.members: dict[int, object] = {}

    def close(self):
        if getattr(self, "h", None):
            A.lib().slbm_pool_free(self.h)
            self.h = None
            self.members.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, dom) -> int:
        slot = C.c_int32()
        A.check(A.lib().slbm_pool_add(self.h, dom.h, C.byref(slot)))
        self.members[slot.value] = dom
        return slot.value

    def remove(self, slot: int):
        A.check(A.lib().slbm_pool_remove(self.h, int(slot)))
        self.members.pop(slot, None)

    def step(self, k: int = 1, graph: bool = True):
        A.check(A.lib().slbm_pool_step(self.h, int(k), int(bool(graph))))

    def reduce(self) -> np.ndarray:
        """(capacity, 5) FP64 sums per slot; zeros for free slots."""
        out = np.zeros((self.capacity, 5))
        A.check(A.lib().slbm_pool_reduce(self.h, out.ctypes.data, A.MEM_HOST))
        return out

    def reduce_device(self, out):
        A.check(A.lib().slbm_pool_reduce(self.h, out.data_ptr(), A.MEM_DEVICE))

    def reduce_ext(self) -> np.ndarray:
        """(capacity, 7): the five sums plus max |f_i - w_i| and max |u| per
        slot; zeros for free slots."""
        out = np.zeros((self.capacity, 7))
        A.check(A.lib().slbm_pool_reduce_ext(self.h, out.ctypes.data, A.MEM_HOST))
        return out

    def reduce_ext_device(self, out):
        A.check(A.lib().slbm_pool_reduce_ext(self.h, out.data_ptr(), A.MEM_DEVICE))

    def set_launch(self, threads: int, ctas_per_sm: int = 0):
        A.check(A.lib().slbm_pool_set_launch(self.h, int(threads), int(ctas_per_sm)))

    def set_split(self, split_cells: int):
        """Members with >= split_cells fluid cells step with their own kernels
        inside the pool's launch sequence; 0 batches every member."""
        A.check(A.lib().slbm_pool_set_split(self.h, int(split_cells)))

    def set_group_bytes(self, nbytes: int):
        """Batched members run in groups of at most nbytes of state + index,
        each group all k steps of a `step(k)` before the next (L2 reuse);
        0 = one group."""
        A.check(A.lib().slbm_pool_set_group_bytes(self.h, int(nbytes)))

    def set_streams(self, n: int):
        """Graph steps spread the large members over n streams (forked from
        and joined into the pool's stream); 1 = all in order."""
        A.check(A.lib().slbm_pool_set_streams(self.h, int(n)))

    def abort(self, raise_flag: bool = True):
        A.check(A.lib().slbm_pool_abort(self.h, int(bool(raise_flag))))
