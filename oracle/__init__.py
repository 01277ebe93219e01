"""Plain CPU oracle for the checkerboard Metropolis sweep (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``isg_oracle.c`` (one int8 per
spin, the paper's definitions written out plainly) through ctypes and shares no
code with the CUDA library in ``paper_1411_0127_gb300``.

Passages followed (arXiv:1411.0127): Eq. (1) Hamiltonian, Eq. (2) bimodal
couplings, Sec. 1 checkerboard colours, Sec. 4 Metropolis rule and integer
threshold comparison, Sec. 3 MINSTD, MT19937 and Parisi-Rapuano.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isg_oracle.c")
_HDR = os.path.join(_HERE, "isg_oracle.h")
_LIB = os.path.join(_HERE, "libisg_oracle.so")

RNG_MINSTD = 0
RNG_MT19937 = 1
RNG_PR = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: same results on x86 and Arm)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None
_override = None   # path of another build of isg_oracle.c to bind instead (tests)


def use_library(path):
    """Bind the wrapper to another build of isg_oracle.c (None: the default build).
    The mutation tests use this to check that the pins catch planted mistakes."""
    global _lib, _override
    _lib, _override = None, path


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_override or build())
        u64, i64, i32, u32, dbl = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_uint32, ctypes.c_double)
        vp = ctypes.c_void_p
        sig = {
            "or_splitmix64": (u64, [u64, u64]),
            "or_thresholds": (None, [dbl, vp]),
            "or_rows_per_stream": (i64, [i32]),
            "or_num_streams": (i64, [i32]),
            "or_mt19937_outputs": (None, [u32, vp, i64]),
            "or_minstd_outputs": (None, [u32, vp, i64]),
            "or_pr_outputs": (None, [u64, vp, i64]),
            "or_initial_spin": (i32, [u64, i64]),
            "or_initial_coupling": (i32, [u64, i64, i32]),
            "or_stream_word": (u64, [u64, i64]),
            "or_unsatisfied": (i32, [ctypes.c_int8, vp, vp]),
            "or_accept": (i32, [i32, u32, vp]),
            "or_create": (vp, [i32, u64, u64, dbl, i32]),
            "or_create2": (vp, [i32, u64, u64, u64, dbl, i32]),
            "or_destroy": (None, [vp]),
            "or_sweep": (None, [vp, i64, i32]),
            "or_energy": (i64, [vp]),
            "or_tracked_energy": (i64, [vp]),
            "or_overlap": (i64, [vp, vp]),
            "or_hash": (u64, [vp]),
            "or_draws_per_stream_done": (i64, [vp, i64]),
            "or_get_spins": (None, [vp, vp]),
            "or_set_spins": (None, [vp, vp]),
            "or_get_couplings": (None, [vp, vp]),
            "or_set_couplings": (None, [vp, vp]),
            "or_move_counts": (None, [vp, vp, vp]),
            "or_acceptance_trial": (None, [i32, u32, dbl, i64, vp]),
            "or_peek_draws": (None, [vp, i64, i64, vp]),
            "or_pass_range": (None, [vp, i32, i64, i64, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def splitmix64(seed: int, n: int) -> int:
    return int(lib().or_splitmix64(seed & (2**64 - 1), n))


def thresholds(beta: float) -> np.ndarray:
    t = np.zeros(4, dtype=np.uint32)
    lib().or_thresholds(float(beta), _ptr(t))
    return t


def rows_per_stream(L: int) -> int:
    return int(lib().or_rows_per_stream(L))


def num_streams(L: int) -> int:
    return int(lib().or_num_streams(L))


def mt19937_outputs(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    lib().or_mt19937_outputs(seed & 0xFFFFFFFF, _ptr(out), n)
    return out


def minstd_outputs(x0: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    lib().or_minstd_outputs(x0, _ptr(out), n)
    return out


def pr_outputs(v: int, n: int) -> np.ndarray:
    """Parisi-Rapuano outputs from seed word v (see or_pr_outputs)."""
    out = np.empty(n, dtype=np.uint32)
    lib().or_pr_outputs(v & (2**64 - 1), _ptr(out), n)
    return out


def initial_spin(seed_spin: int, i: int) -> int:
    """Spin of site i as or_create draws it (Eq. (2))."""
    return int(lib().or_initial_spin(seed_spin & (2**64 - 1), int(i)))


def initial_coupling(seed_J: int, i: int, d: int) -> int:
    """Coupling J[d][i] (bond from site i to its +d neighbour) as or_create draws it."""
    return int(lib().or_initial_coupling(seed_J & (2**64 - 1), int(i), int(d)))


def stream_word(seed_rng: int, t: int) -> int:
    """64-bit seed word of RNG stream t (see or_stream_word)."""
    return int(lib().or_stream_word(seed_rng & (2**64 - 1), int(t)))


def unsatisfied(s: int, nb, J) -> int:
    nb = np.ascontiguousarray(nb, dtype=np.int8)
    J = np.ascontiguousarray(J, dtype=np.int8)
    return int(lib().or_unsatisfied(int(s), _ptr(nb), _ptr(J)))


def acceptance_trial(kind: int, seed: int, beta: float, n: int) -> np.ndarray:
    """Accepted counts out of n decisions for u = 0, 1, 2 (one stream's draws)."""
    out = np.zeros(3, dtype=np.int64)
    lib().or_acceptance_trial(kind, seed, float(beta), n, _ptr(out))
    return out


def accept(u: int, d: int, thr: np.ndarray) -> bool:
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    return bool(lib().or_accept(int(u), int(d), _ptr(thr)))


class OracleSim:
    """One lattice with its coupling sample, spins and RNG streams."""

    def __init__(self, L: int, seed_J: int, seed_spin: int, beta: float, kind: int, seed_rng: int = None):
        if seed_rng is None:
            self._h = lib().or_create(L, seed_J, seed_spin, float(beta), kind)
        else:
            self._h = lib().or_create2(L, seed_J, seed_spin, seed_rng, float(beta), kind)
        if not self._h:
            raise ValueError("oracle: invalid arguments L=%r beta=%r kind=%r" % (L, beta, kind))
        self.L, self.N, self.kind, self.beta = L, L ** 3, kind, beta

    def close(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    __del__ = close

    def sweep(self, n: int = 1, threads: int = 1):
        lib().or_sweep(self._h, n, threads)

    def pass_range(self, colour: int, t0: int, t1: int, threads: int = 1):
        """One colour pass over streams [t0, t1) only (timing samples)."""
        lib().or_pass_range(self._h, colour, t0, t1, threads)

    def energy(self) -> int:
        return int(lib().or_energy(self._h))

    def tracked_energy(self) -> int:
        return int(lib().or_tracked_energy(self._h))

    def overlap(self, other: "OracleSim") -> int:
        return int(lib().or_overlap(self._h, other._h))

    def hash(self) -> int:
        return int(lib().or_hash(self._h))

    def draws_done(self, t: int) -> int:
        return int(lib().or_draws_per_stream_done(self._h, t))

    def peek_draws(self, t: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint32)
        lib().or_peek_draws(self._h, t, n, _ptr(out))
        return out

    def move_counts(self):
        att = np.zeros(7, dtype=np.int64)
        acc = np.zeros(7, dtype=np.int64)
        lib().or_move_counts(self._h, _ptr(att), _ptr(acc))
        return att, acc

    def spins(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int8)
        lib().or_get_spins(self._h, _ptr(out))
        return out

    def set_spins(self, s: np.ndarray):
        s = np.ascontiguousarray(s, dtype=np.int8).reshape(-1)
        assert s.size == self.N
        lib().or_set_spins(self._h, _ptr(s))

    def couplings(self) -> np.ndarray:
        out = np.empty(3 * self.N, dtype=np.int8)
        lib().or_get_couplings(self._h, _ptr(out))
        return out.reshape(3, self.N)

    def set_couplings(self, J: np.ndarray):
        J = np.ascontiguousarray(J, dtype=np.int8).reshape(-1)
        assert J.size == 3 * self.N
        lib().or_set_couplings(self._h, _ptr(J))


def stream_draws(kind: int, word: int, n: int) -> np.ndarray:
    """The first n draws of a stream with seed word `word`, as the Metropolis
    rule compares them (Sec. 4): MT19937 and Parisi-Rapuano outputs as they are,
    MINSTD states doubled (d = 2x)."""
    if kind == RNG_MT19937:
        return mt19937_outputs(word & 0xFFFFFFFF, n)
    if kind == RNG_PR:
        return pr_outputs(word, n)
    return (minstd_outputs(1 + word % (2**31 - 2), n).astype(np.uint64) << 1).astype(np.uint32)


class SampledFirstSweep:
    """The spins after the first sweep from the initial state, one site at a time,
    for lattices too large to hold (L = 2048 is 34 GB as OracleSim's int8
    arrays).  It takes the same steps as OracleSim in the order the method fixes:
    the red pass (colour 0) reads only initial blue spins, the blue pass reads the
    red spins after the red pass; a site of colour c in row r = y + L z owned by
    stream t = r // R uses draw number (r - t R) L/2 + x // 2 of that stream's
    pass of colour c, the blue pass starting after the red pass's rows_t L/2
    draws (Sec. 1 checkerboard; Sec. 4 rule with u unsatisfied bonds)."""

    def __init__(self, L: int, seed_J: int, seed_spin: int, beta: float, kind: int, seed_rng: int = None):
        self.L, self.seed_J, self.seed_spin, self.kind = L, seed_J, seed_spin, kind
        self.seed_rng = seed_spin if seed_rng is None else seed_rng
        self.R, self.S = rows_per_stream(L), num_streams(L)
        self.thr = thresholds(beta)
        self._draws = {}   # (stream, draw number) -> draw

    def _rows(self, t: int) -> int:
        return min(self.R, self.L * self.L - t * self.R)

    def _tk(self, x: int, y: int, z: int):
        """(stream, draw number in sweep 1) of the attempt at site (x, y, z)."""
        L = self.L
        c = (x + y + z) & 1
        r = (y % L) + L * (z % L)
        t = r // self.R
        return t, (r - t * self.R) * (L // 2) + (x % L) // 2 + c * self._rows(t) * (L // 2)

    def _fetch(self, need: dict):
        """Generate each stream once, up to the largest draw number asked of it,
        and keep only the draws asked for."""
        for t, ks in need.items():
            d = stream_draws(self.kind, stream_word(self.seed_rng, t), max(ks) + 1)
            for k in ks:
                self._draws[(t, k)] = int(d[k])

    def _draw(self, t: int, k: int) -> int:
        if (t, k) not in self._draws:
            self._fetch({t: {k}})
        return self._draws[(t, k)]

    def prefetch(self, sites):
        """Fetch the draws that after() needs for these sites, one generator run
        per stream (memory stays at one stream's draws)."""
        need = {}
        for x, y, z in sites:
            updates = [(x, y, z)]
            if (x + y + z) & 1:
                updates += [(x + 1, y, z), (x - 1, y, z), (x, y + 1, z), (x, y - 1, z), (x, y, z + 1), (x, y, z - 1)]
            for u in updates:
                t, k = self._tk(*u)
                need.setdefault(t, set()).add(k)
        self._fetch(need)

    def _i(self, x: int, y: int, z: int) -> int:
        L = self.L
        return (x % L) + L * (y % L) + L * L * (z % L)

    def initial(self, x: int, y: int, z: int) -> int:
        return initial_spin(self.seed_spin, self._i(x, y, z))

    def _update(self, x: int, y: int, z: int, nbspin) -> int:
        L, sJ = self.L, self.seed_J
        s = self.initial(x, y, z)
        nb = [nbspin(x + 1, y, z), nbspin(x - 1, y, z), nbspin(x, y + 1, z),
              nbspin(x, y - 1, z), nbspin(x, y, z + 1), nbspin(x, y, z - 1)]
        Jb = [initial_coupling(sJ, self._i(x, y, z), 0), initial_coupling(sJ, self._i(x - 1, y, z), 0),
              initial_coupling(sJ, self._i(x, y, z), 1), initial_coupling(sJ, self._i(x, y - 1, z), 1),
              initial_coupling(sJ, self._i(x, y, z), 2), initial_coupling(sJ, self._i(x, y, z - 1), 2)]
        u = unsatisfied(s, nb, Jb)
        return -s if accept(u, self._draw(*self._tk(x, y, z)), self.thr) else s

    def red(self, x: int, y: int, z: int) -> int:
        """Spin of a colour-0 site after the red pass of sweep 1."""
        return self._update(x, y, z, self.initial)

    def after(self, x: int, y: int, z: int) -> int:
        """Spin of any site after sweep 1."""
        if (x + y + z) & 1 == 0:
            return self.red(x, y, z)
        return self._update(x, y, z, self.red)

