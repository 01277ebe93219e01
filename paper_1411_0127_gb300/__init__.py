"""Python binding of ``libisg.so``, the GB300 checkerboard Metropolis engine for
the 3D Edwards-Anderson +-J spin glass (arXiv:1411.0127).

This module only marshals arguments to the C-ABI declared in ``include/isg.h``;
every step of the sweep runs in the CUDA kernels of ``csrc/``.  PyTorch, when
present, provides the device allocator (its caching allocator) and streams.
If ``libisg.so`` is missing the import of the library fails loudly: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libisg.so")

ISG_OK, ISG_ERR_ARG, ISG_ERR_NOMEM, ISG_ERR_CUDA, ISG_ERR_TIMEOUT, ISG_ERR_MISMATCH, ISG_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6
ISG_RNG_MINSTD, ISG_RNG_MT19937, ISG_RNG_PARISI_RAPUANO = 0, 1, 2
RNG_KINDS = {"minstd": ISG_RNG_MINSTD, "mt19937": ISG_RNG_MT19937, "parisi_rapuano": ISG_RNG_PARISI_RAPUANO}

_vp, _i32, _i64, _u64, _dbl, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                    ctypes.c_double, ctypes.c_size_t)
_PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); every name here is declared in include/isg.h
SIGNATURES = {
    "isg_create": (_i32, [_i32, _u64, _u64, _dbl, _i32, _PP]),
    "isg_create2": (_i32, [_i32, _u64, _u64, _u64, _dbl, _i32, _PP]),
    "isg_destroy": (None, [_vp]),
    "isg_set_allocator": (_i32, [_vp, _vp, _vp]),
    "isg_last_error": (ctypes.c_char_p, []),
    "isg_info": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "isg_sweep": (_i32, [_vp, _i64, _vp]),
    "isg_sweep_plain": (_i32, [_vp, _i64, _vp]),
    "isg_sweeps_done": (_i32, [_vp, _vp]),
    "isg_sweep_info": (_i32, [_vp, _vp]),
    "isg_energy": (_i32, [_vp, _vp, _vp]),
    "isg_tracked_energy": (_i32, [_vp, _vp]),
    "isg_overlap": (_i32, [_vp, _vp, _vp, _vp]),
    "isg_hash": (_i32, [_vp, _vp, _vp]),
    "isg_read_spins": (_i32, [_vp, _vp, _sz, _vp]),
    "isg_write_spins": (_i32, [_vp, _vp, _sz, _vp]),
    "isg_read_spins_packed": (_i32, [_vp, _vp, _sz, _vp]),
    "isg_write_spins_packed": (_i32, [_vp, _vp, _sz, _vp]),
    "isg_exchange_async": (_i32, [_vp, _vp, _vp, _sz, _i64, _vp, _vp]),
    "isg_read_couplings": (_i32, [_vp, _vp, _sz, _vp]),
    "isg_write_couplings": (_i32, [_vp, _vp, _sz, _vp]),
    "isg_save": (_i32, [_vp, _vp, _vp, _vp]),
    "isg_load": (_i32, [_vp, _sz, _PP]),
    "isg_stencil_decisions": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "isg_peek_draws": (_i32, [_vp, _i64, _i64, _vp]),
    "isg_batch_test_stall": (_i32, [_vp]),
    "isg_sweep_test_stall": (_i32, [_vp]),
    "isg_energy_static_scratch": (_i32, [_vp, _vp, _vp]),
    "isg_batch_create": (_i32, [_i32, _vp, _vp, _vp, _vp, _i32, _PP]),
    "isg_batch_destroy": (None, [_vp]),
    "isg_batch_info": (_i32, [_vp, _vp, _vp, _vp]),
    "isg_batch_member": (_i32, [_vp, _i32, _PP]),
    "isg_batch_set_config": (_i32, [_vp, _i32, _i32, _i32, _i32]),
    "isg_batch_get_config": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "isg_batch_run": (_i32, [_vp, _i64, _i32, _vp]),
    "isg_batch_measure": (_i32, [_vp, _vp, _vp, _vp]),
    "isg_batch_tracked": (_i32, [_vp, _vp, _vp, _vp]),
    "isg_server_create": (_i32, [_sz, _i32, _i32, _PP]),
    "isg_server_destroy": (None, [_vp]),
    "isg_server_submit": (_i32, [_vp, _i32, _u64, _u64, _dbl, _i32, _i64, _dbl, _vp]),
    "isg_server_run": (_i32, [_vp, _dbl]),
    "isg_server_job": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "isg_server_stats": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "isg_rng_count_odd": (_i32, [_i32, _u64, _i64, _i64, _vp, _vp]),
    "isg_int_rate": (_i32, [_i32, _vp]),
    "isg_amsc_create": (_i32, [_i32, _vp, _vp, _u64, _dbl, _i32, _PP]),
    "isg_amsc_destroy": (None, [_vp]),
    "isg_amsc_sweep": (_i32, [_vp, _i64, _vp]),
    "isg_amsc_energies": (_i32, [_vp, _vp, _vp]),
    "isg_amsc_info": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "isg_amsc_read_spins": (_i32, [_vp, _i32, _vp, _sz, _vp]),
}


def rng_count_odd(rng_kind, seed: int, streams: int, n: int):
    """Odd raw outputs of `streams` generator streams of n numbers each, and the
    generation kernel's device time in ms (see isg_rng_count_odd)."""
    kind = RNG_KINDS[rng_kind] if isinstance(rng_kind, str) else int(rng_kind)
    odd, ms = ctypes.c_uint64(), ctypes.c_double()
    _check(lib().isg_rng_count_odd(kind, int(seed) & (2**64 - 1), int(streams), int(n), ctypes.byref(odd),
                                   ctypes.byref(ms)))
    return odd.value, ms.value


def int_rate(mode: int) -> float:
    """32-bit integer ops/s on independent chains (0: LOP3 + IMAD, 1: LOP3, 2: IMAD)."""
    v = ctypes.c_double()
    _check(lib().isg_int_rate(int(mode), ctypes.byref(v)))
    return v.value


class IsgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("isg error %d: %s" % (code, msg))
        self.code = code


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Load libisg.so (built by ``__graft_entry__.build()``); raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libisg.so is not built (%s); run `python -c 'import __graft_entry__ as g; "
                               "g.build()'` -- there is no CPU fallback" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != ISG_OK:
        raise IsgError(rc, lib().isg_last_error().decode(errors="replace"))


def _stream(stream) -> int:
    """cudaStream_t of a torch stream, an int handle, or the current torch stream."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ------------------------------------------------------------- allocator ---
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_keep = []


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    import torch

    def _alloc(size, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size))
        except Exception:
            return None

    def _free(ptr, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_T(_alloc), _FREE_T(_free)
    _keep[:] = [a, f]
    _check(lib().isg_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))


def use_default_allocator():
    _check(lib().isg_set_allocator(None, None, None))


# ---------------------------------------------------------------- handle ---
class Sim:
    """One L^3 lattice (one replica): couplings, bit-packed spins, RNG streams."""

    def __init__(self, L: int, seed_J: int, seed_spin: int, beta: float, rng_kind="minstd", *, seed_rng=None,
                 _handle=None):
        kind = RNG_KINDS[rng_kind] if isinstance(rng_kind, str) else int(rng_kind)
        if _handle is None:
            h = ctypes.c_void_p()
            if seed_rng is None:
                _check(lib().isg_create(int(L), int(seed_J) & (2**64 - 1), int(seed_spin) & (2**64 - 1),
                                        float(beta), kind, ctypes.byref(h)))
            else:
                _check(lib().isg_create2(int(L), int(seed_J) & (2**64 - 1), int(seed_spin) & (2**64 - 1),
                                         int(seed_rng) & (2**64 - 1), float(beta), kind, ctypes.byref(h)))
            _handle = h.value
        self._h = _handle
        self.L, self.N, self.kind, self.beta = int(L), int(L) ** 3, kind, float(beta)

    @property
    def handle(self) -> int:
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().isg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        L, wb, W = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        S, R = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().isg_info(self._h, ctypes.byref(L), ctypes.byref(wb), ctypes.byref(W), ctypes.byref(S),
                              ctypes.byref(R)))
        return {"L": L.value, "word_bits": wb.value, "words_per_row": W.value, "streams": S.value,
                "rows_per_stream": R.value}

    def sweep(self, n: int = 1, stream=None):
        """Enqueue n sweeps (isg_sweep).  Calls of 8 or more sweeps on large MINSTD
        and MT19937 lattices run as persistent multi-pass launches (see
        passes_per_launch); the trajectory is the same either way."""
        _check(lib().isg_sweep(self._h, int(n), _stream(stream)))

    def sweep_plain(self, n: int = 1, stream=None):
        _check(lib().isg_sweep_plain(self._h, int(n), _stream(stream)))

    def passes_per_launch(self) -> int:
        """128 if isg_sweep runs this lattice's passes in persistent launches of up
        to 64 sweeps, 1 if it launches every colour pass on its own."""
        v = ctypes.c_int()
        _check(lib().isg_sweep_info(self._h, ctypes.byref(v)))
        return v.value

    def sweeps_done(self) -> int:
        v = ctypes.c_int64()
        _check(lib().isg_sweeps_done(self._h, ctypes.byref(v)))
        return v.value

    def energy(self, stream=None) -> int:
        v = ctypes.c_int64()
        _check(lib().isg_energy(self._h, ctypes.byref(v), _stream(stream)))
        return v.value

    def tracked_energy(self) -> int:
        v = ctypes.c_int64()
        _check(lib().isg_tracked_energy(self._h, ctypes.byref(v)))
        return v.value

    def overlap(self, other: "Sim", stream=None) -> int:
        v = ctypes.c_int64()
        _check(lib().isg_overlap(self._h, other._h, ctypes.byref(v), _stream(stream)))
        return v.value

    def hash(self, stream=None) -> int:
        v = ctypes.c_uint64()
        _check(lib().isg_hash(self._h, ctypes.byref(v), _stream(stream)))
        return v.value

    def read_spins(self, stream=None, out: np.ndarray = None) -> np.ndarray:
        """Spins as int8 +-1 in site order.  `out` (C-contiguous int8, at least
        L^3 values; pinned memory for full copy speed) receives them directly."""
        if out is None:
            out = np.empty(self.N, dtype=np.int8)
        elif out.dtype != np.int8 or not out.flags["C_CONTIGUOUS"] or out.size < self.N:
            raise ValueError("out must be a C-contiguous int8 array of at least L^3 values")
        _check(lib().isg_read_spins(self._h, _ptr(out), out.size, _stream(stream)))
        return out

    def read_spins_packed(self, stream=None, out: np.ndarray = None) -> np.ndarray:
        """Spins as packed bits (uint8, ceil(L^3/8) bytes): bit i & 7 of byte i >> 3
        is site i, 1 meaning +1 (numpy.unpackbits(..., bitorder="little"))."""
        nb = (self.N + 7) // 8
        if out is None:
            out = np.empty(nb, dtype=np.uint8)
        elif out.dtype != np.uint8 or not out.flags["C_CONTIGUOUS"] or out.size < nb:
            raise ValueError("out must be a C-contiguous uint8 array of at least ceil(L^3/8) bytes")
        _check(lib().isg_read_spins_packed(self._h, _ptr(out), out.size, _stream(stream)))
        return out

    def write_spins_packed(self, bits: np.ndarray, stream=None):
        bits = np.ascontiguousarray(bits, dtype=np.uint8).reshape(-1)
        _check(lib().isg_write_spins_packed(self._h, _ptr(bits), bits.size, _stream(stream)))

    def exchange_async(self, bits_in: np.ndarray = None, bits_out: np.ndarray = None, sweeps: int = 1,
                       E_out: np.ndarray = None, stream=None):
        """Enqueue, without synchronising: packed spins in (optional), `sweeps`
        sweeps, packed spins out and the tracked energy into E_out[0] (optional;
        int64).  The arrays must be C-contiguous, should be pinned (torch's
        pin_memory) for the copies to overlap other work, and must be kept (and
        bits_in left unchanged) until the stream has passed this call."""
        nb = (self.N + 7) // 8
        for a in (bits_in, bits_out):
            if a is not None and (a.dtype != np.uint8 or not a.flags["C_CONTIGUOUS"] or a.size < nb):
                raise ValueError("bit buffers must be C-contiguous uint8 arrays of at least ceil(L^3/8) bytes")
        if E_out is not None and (E_out.dtype != np.int64 or not E_out.flags["C_CONTIGUOUS"] or E_out.size < 1):
            raise ValueError("E_out must be a C-contiguous int64 array")
        _check(lib().isg_exchange_async(self._h, None if bits_in is None else _ptr(bits_in),
                                        None if bits_out is None else _ptr(bits_out), nb, int(sweeps),
                                        None if E_out is None else _ptr(E_out), _stream(stream)))

    def write_spins(self, s: np.ndarray, stream=None):
        s = np.ascontiguousarray(s, dtype=np.int8).reshape(-1)
        _check(lib().isg_write_spins(self._h, _ptr(s), s.size, _stream(stream)))

    def read_couplings(self, stream=None) -> np.ndarray:
        out = np.empty(3 * self.N, dtype=np.int8)
        _check(lib().isg_read_couplings(self._h, _ptr(out), out.size, _stream(stream)))
        return out.reshape(3, self.N)

    def write_couplings(self, J: np.ndarray, stream=None):
        J = np.ascontiguousarray(J, dtype=np.int8).reshape(-1)
        _check(lib().isg_write_couplings(self._h, _ptr(J), J.size, _stream(stream)))

    def save(self, stream=None) -> bytes:
        n = ctypes.c_size_t(0)
        _check(lib().isg_save(self._h, None, ctypes.byref(n), _stream(stream)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().isg_save(self._h, buf, ctypes.byref(n), _stream(stream)))
        return buf.raw[:n.value]

    @classmethod
    def load(cls, data: bytes) -> "Sim":
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(data, len(data))
        _check(lib().isg_load(buf, len(data), ctypes.byref(h)))
        sim = cls.__new__(cls)
        sim._h = h.value
        L = ctypes.c_int()
        _check(lib().isg_info(sim._h, ctypes.byref(L), None, None, None, None))
        sim.L, sim.N = L.value, L.value ** 3
        sim.kind, sim.beta = None, None
        return sim

    def peek_draws(self, t: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint32)
        _check(lib().isg_peek_draws(self._h, int(t), int(n), _ptr(out)))
        return out


def stencil_decisions(codes: np.ndarray, draws: np.ndarray, thr) -> tuple[np.ndarray, np.ndarray]:
    """Device bit logic on explicit stencils (see isg_stencil_decisions)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    draws = np.ascontiguousarray(draws, dtype=np.uint32)
    t = np.ascontiguousarray(thr, dtype=np.uint32)
    assert codes.size == draws.size and t.size == 3
    flip = np.empty(codes.size, dtype=np.uint8)
    u = np.empty(codes.size, dtype=np.uint8)
    _check(lib().isg_stencil_decisions(_ptr(codes), _ptr(draws), codes.size, _ptr(t), _ptr(flip), _ptr(u)))
    return flip, u


class _Member(Sim):
    """A replica owned by a Batch (never destroyed through this object)."""

    def close(self):
        self._h = None


class Batch:
    """Many samples of uneven L, two replicas each, swept by persistent launches."""

    def __init__(self, L, seed_J, seed_spin, beta, rng_kind="mt19937"):
        kind = RNG_KINDS[rng_kind] if isinstance(rng_kind, str) else int(rng_kind)
        n = len(L)
        La = np.ascontiguousarray(L, dtype=np.int32)
        J = np.ascontiguousarray([int(v) & (2**64 - 1) for v in seed_J], dtype=np.uint64)
        S = np.ascontiguousarray([int(v) & (2**64 - 1) for v in seed_spin], dtype=np.uint64)
        B = np.ascontiguousarray(beta, dtype=np.float64)
        assert J.size == n and S.size == 2 * n and B.size == n
        h = ctypes.c_void_p()
        _check(lib().isg_batch_create(n, _ptr(La), _ptr(J), _ptr(S), _ptr(B), kind, ctypes.byref(h)))
        self._h = h.value
        self.n, self.kind = n, kind
        self.L = [int(v) for v in La]
        self.beta = [float(v) for v in B]
        self._args = (list(self.L), [int(v) for v in J], [int(v) for v in S], list(self.beta), kind)

    def set_config(self, shape: int, capacity: int = 0, resident: int = 1, words_per_lane: int = 1):
        """Execution configuration (see isg_batch_set_config); results do not depend on it."""
        _check(lib().isg_batch_set_config(self._h, int(shape), int(capacity), int(resident), int(words_per_lane)))

    def get_config(self) -> tuple:
        """(shape, capacity, resident, words_per_lane)."""
        a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().isg_batch_get_config(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(d)))
        return a.value, b.value, c.value, d.value

    def twin(self) -> "Batch":
        """A new batch with the same samples, seeds, temperatures and kind, at
        sweep 0 (the autotuner times candidates on one)."""
        L, J, S, B, kind = self._args
        return Batch(L, J, S, B, kind)

    def autotune(self, sweeps: int = 8, cache: str = None, stream=None) -> dict:
        """Choose the fastest execution configuration (paper_1411_0127_gb300.autotune)
        and apply it; the batch's own state is not touched."""
        from . import autotune as _at
        res = _at.tune(self, sweeps=sweeps, cache=cache, stream=stream)
        self.set_config(*res["config"])
        return res

    def close(self):
        if getattr(self, "_h", None):
            lib().isg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        s, b, a = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().isg_batch_info(self._h, ctypes.byref(s), ctypes.byref(b), ctypes.byref(a)))
        return {"samples": s.value, "bundles": b.value, "attempts_per_sweep": a.value}

    def run(self, sweeps: int, group_sweeps: int = 64, stream=None):
        _check(lib().isg_batch_run(self._h, int(sweeps), int(group_sweeps), _stream(stream)))

    def member(self, i: int) -> Sim:
        h = ctypes.c_void_p()
        _check(lib().isg_batch_member(self._h, int(i), ctypes.byref(h)))
        m = _Member.__new__(_Member)
        m._h = h.value
        m.L = self.L[i // 2]
        m.N = m.L ** 3
        m.kind, m.beta = self.kind, self.beta[i // 2]
        return m

    def measure(self, stream=None):
        E = np.empty(2 * self.n, dtype=np.int64)
        Q = np.empty(self.n, dtype=np.int64)
        _check(lib().isg_batch_measure(self._h, _ptr(E), _ptr(Q), _stream(stream)))
        return E, Q

    def tracked(self, stream=None):
        E = np.empty(2 * self.n, dtype=np.int64)
        H = np.empty(2 * self.n, dtype=np.uint64)
        _check(lib().isg_batch_tracked(self._h, _ptr(E), _ptr(H), _stream(stream)))
        return E, H


class Amsc:
    """32 systems of one size in asynchronous multispin coding (one shared draw
    per site); system b follows Sim(L, seed_J[b], seed_spin[b], beta, kind,
    seed_rng=seed_rng) bit for bit."""

    SAMPLES = 32

    def __init__(self, L: int, seed_J, seed_spin, seed_rng: int, beta: float, rng_kind="mt19937"):
        kind = RNG_KINDS[rng_kind] if isinstance(rng_kind, str) else int(rng_kind)
        J = np.ascontiguousarray([int(v) & (2**64 - 1) for v in seed_J], dtype=np.uint64)
        S = np.ascontiguousarray([int(v) & (2**64 - 1) for v in seed_spin], dtype=np.uint64)
        if J.size != self.SAMPLES or S.size != self.SAMPLES:
            raise ValueError("Amsc needs 32 coupling seeds and 32 spin seeds")
        h = ctypes.c_void_p()
        _check(lib().isg_amsc_create(int(L), _ptr(J), _ptr(S), int(seed_rng) & (2**64 - 1), float(beta), kind,
                                     ctypes.byref(h)))
        self._h = h.value
        self.L, self.N, self.kind, self.beta = int(L), int(L) ** 3, kind, float(beta)

    def close(self):
        if getattr(self, "_h", None):
            lib().isg_amsc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n: int = 1, stream=None):
        _check(lib().isg_amsc_sweep(self._h, int(n), _stream(stream)))

    def info(self) -> dict:
        """Size, RNG streams, rows per stream and the sweep kernel's form on the
        current device (0: staged by bulk copies; 4 or 8: register form with
        that many blocks of 32 sites in flight per lane)."""
        L, nb = ctypes.c_int(), ctypes.c_int()
        S, R = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().isg_amsc_info(self._h, ctypes.byref(L), ctypes.byref(S), ctypes.byref(R), ctypes.byref(nb)))
        return {"L": L.value, "streams": S.value, "rows_per_stream": R.value, "form": nb.value}

    def energies(self, stream=None) -> np.ndarray:
        E = np.empty(self.SAMPLES, dtype=np.int64)
        _check(lib().isg_amsc_energies(self._h, _ptr(E), _stream(stream)))
        return E

    def spins(self, sample: int, stream=None) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int8)
        _check(lib().isg_amsc_read_spins(self._h, int(sample), _ptr(out), out.size, _stream(stream)))
        return out


class Server:
    """Continuous-batching request server for quench jobs (see isg_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 150 * 10**9, quantum_sweeps: int = 64, max_active: int = 4096):
        h = ctypes.c_void_p()
        _check(lib().isg_server_create(int(hbm_budget_bytes), int(quantum_sweeps), int(max_active),
                                       ctypes.byref(h)))
        self._h = h.value

    def close(self):
        if getattr(self, "_h", None):
            lib().isg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, L, seed_J, seed_spin, beta, rng_kind, sweeps, arrival_s=0.0) -> int:
        kind = RNG_KINDS[rng_kind] if isinstance(rng_kind, str) else int(rng_kind)
        jid = ctypes.c_int64()
        _check(lib().isg_server_submit(self._h, int(L), int(seed_J) & (2**64 - 1), int(seed_spin) & (2**64 - 1),
                                       float(beta), kind, int(sweeps), float(arrival_s), ctypes.byref(jid)))
        return jid.value

    def run(self, time_limit_s: float = 0.0):
        _check(lib().isg_server_run(self._h, float(time_limit_s)))

    def job(self, jid: int) -> dict:
        st, E, H = ctypes.c_int(), ctypes.c_int64(), ctypes.c_uint64()
        a, ad, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().isg_server_job(self._h, int(jid), ctypes.byref(st), ctypes.byref(E), ctypes.byref(H),
                                    ctypes.byref(a), ctypes.byref(ad), ctypes.byref(d)))
        return {"status": st.value, "E": E.value, "H": H.value, "arrival": a.value, "admit": ad.value,
                "done": d.value, "latency": d.value - a.value}

    def stats(self) -> dict:
        it, at = ctypes.c_int64(), ctypes.c_int64()
        wall, busy = ctypes.c_double(), ctypes.c_double()
        pa, pb = ctypes.c_int(), ctypes.c_size_t()
        _check(lib().isg_server_stats(self._h, ctypes.byref(it), ctypes.byref(at), ctypes.byref(wall),
                                      ctypes.byref(busy), ctypes.byref(pa), ctypes.byref(pb)))
        return {"iterations": it.value, "attempts": at.value, "wall_s": wall.value, "busy_s": busy.value,
                "peak_active": pa.value, "peak_bytes": pb.value}
