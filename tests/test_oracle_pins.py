"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test names what fixes the expected value: a published generator output, a
library routine, a closed form, an invariant of the dynamics or brute force over
tiny inputs (arXiv:1411.0127 passages cited per test).
"""
import math
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import OracleSim, RNG_MINSTD, RNG_MT19937, RNG_PR

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KINDS = [RNG_MINSTD, RNG_MT19937, RNG_PR]


# --------------------------------------------------------------------------
# Generators (Sec. 3)

def _golden_generators():
    rows = []
    with open(os.path.join(GOLDEN, "generators.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kind, *kv = line.split()
            d = dict(x.split("=") for x in kv)
            rows.append((kind, int(d["seed"], 0), int(d["index"]), int(d["value"], 0)))
    return rows


def test_generator_golden_values():
    rows = _golden_generators()
    assert len(rows) == 4
    for kind, seed, index, value in rows:
        if kind == "mt19937":
            assert int(oracle.mt19937_outputs(seed, index)[-1]) == value
        elif kind == "minstd":
            assert int(oracle.minstd_outputs(seed, index)[-1]) == value
        elif kind == "splitmix64":
            assert oracle.splitmix64(seed, index - 1) == value
        else:
            raise AssertionError(kind)


@pytest.mark.parametrize("seed", [0, 1, 4357, 12345, 2**31 - 1, 2**32 - 1])
def test_mt19937_matches_numpy_legacy_seeding(seed):
    # numpy's legacy RandomState seeding is MT19937's init_genrand(seed).
    bg = np.random.MT19937()
    bg._legacy_seeding(seed)
    ref = bg.random_raw(3000).astype(np.uint32)   # spans several 624-word blocks
    assert np.array_equal(oracle.mt19937_outputs(seed, 3000), ref)


def test_generators_match_cpp_standard_library(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "ref.cpp"
    src.write_text(
        "#include <random>\n#include <cstdio>\n#include <cstdlib>\n"
        "int main(int c, char** v){ unsigned s = (unsigned)strtoul(v[2],0,10); int n = atoi(v[3]);\n"
        " if (v[1][0]=='m') { std::mt19937 g(s); for(int i=0;i<n;i++) printf(\"%u\\n\", (unsigned)g()); }\n"
        " else { std::minstd_rand0 g(s); for(int i=0;i<n;i++) printf(\"%u\\n\", (unsigned)g()); }\n"
        " return 0; }\n")
    exe = tmp_path / "ref"
    subprocess.run([gxx, "-O1", "-o", str(exe), str(src)], check=True)
    for seed in [1, 2, 777, 2**31 - 2]:
        for kind in ["m", "n"]:
            out = subprocess.run([str(exe), kind, str(seed), "2000"], check=True,
                                 capture_output=True, text=True).stdout.split()
            ref = np.array([int(x) for x in out], dtype=np.uint32)
            got = (oracle.mt19937_outputs(seed, 2000) if kind == "m"
                   else oracle.minstd_outputs(seed, 2000))
            assert np.array_equal(got, ref), (kind, seed)


# --------------------------------------------------------------------------
# Integer thresholds (Sec. 4: R < Rmax exp(-beta dE))

def _thr_mp(beta):
    import mpmath
    mpmath.mp.dps = 50
    out = [0]
    for k in (1, 2, 3):
        v = mpmath.mpf(2) ** 32 * mpmath.exp(-4 * k * mpmath.mpf(beta))
        fl = int(mpmath.floor(v))
        # double precision carries ~1e-6 absolute error at 2^32: a value that close
        # to an integer could round either way, so the case must not be used
        if v > 1:
            frac = v - fl
            assert 1e-5 < frac < 1 - 1e-5
        out.append(fl)
    return out


# Parisi-Rapuano (Sec. 3): ira[i] = ira[i-24] + ira[i-55] mod 2^32, R = ira[i] ^ ira[i-61].
# The seeding is a reading of the paper, which gives none: ira[j] = upper 32
# bits of SplitMix64(v, j), j < 61, ira[60] made odd.

def _pr_initial_words(v):
    w = [oracle.splitmix64(v, j) >> 32 for j in range(61)]
    w[60] |= 1
    return w


def _pr_step_matrix():
    """61 x 61 companion matrix of the window (ira[i-61], ..., ira[i-1]) -> the
    window one step later; its last row forms ira[i] from lags 24 and 55."""
    M = np.zeros((61, 61), dtype=object)
    for j in range(60):
        M[j, j + 1] = 1
    M[60, 61 - 24] = 1
    M[60, 61 - 55] = 1
    return M


def _matvec_power(M, n, vec, mod):
    """M^n vec (mod `mod`) by binary powering: a different computation from the
    oracle's ring-buffer iteration."""
    vec = np.array(vec, dtype=object)
    P = M.copy()
    while n:
        if n & 1:
            vec = P.dot(vec) % mod
        n >>= 1
        if n:
            P = P.dot(P) % mod
    return vec


@pytest.mark.parametrize("v", [0, 77, 2**64 - 1])
def test_parisi_rapuano_companion_matrix_powers(v):
    """Output n = ira[61+n] ^ ira[n]: the windows after n and n + 1 steps come
    from powers of the companion matrix mod 2^32, not from iteration."""
    ns = [0, 1, 23, 24, 54, 55, 60, 61, 62, 500, 4099]
    out = oracle.pr_outputs(v, max(ns) + 1)
    s0 = _pr_initial_words(v)
    M = _pr_step_matrix()
    for n in ns:
        a = _matvec_power(M, n, s0, 2**32)
        b = M.dot(a) % 2**32
        assert int(out[n]) == (int(b[60]) ^ int(a[0])), n


def _gf2_mulmod(a, b, p, deg):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a >> deg & 1:
            a ^= p
    return r


def _gf2_xpow(n, p, deg):
    """x^n mod p(x) over GF(2), polynomials as bit masks."""
    r, base = 1, 2
    while n:
        if n & 1:
            r = _gf2_mulmod(r, base, p, deg)
        base = _gf2_mulmod(base, base, p, deg)
        n >>= 1
    return r


def test_parisi_rapuano_low_bits_polynomial_jump():
    """The low bits b_i of ira obey b_i = b_(i-24) ^ b_(i-55) (addition mod 2):
    characteristic polynomial x^55 + x^31 + 1.  Far along the stream (n ~ 10^6)
    the low bit of each output equals b_(61+n) ^ b_n computed by a GF(2)
    polynomial jump from the initial window b_6 .. b_60."""
    v = 2024
    base = 10**6
    out = oracle.pr_outputs(v, base + 40)
    w = _pr_initial_words(v)
    window = [w[6 + j] & 1 for j in range(55)]
    p, deg = (1 << 55) | (1 << 31) | 1, 55

    def bit(i):  # b_i for i >= 6
        c = _gf2_xpow(i - 6, p, deg)
        return sum(window[j] for j in range(55) if c >> j & 1) & 1

    for n in range(base, base + 40):
        assert int(out[n]) & 1 == bit(61 + n) ^ bit(n), n


def test_parisi_rapuano_trinomial_period_structure():
    """x^55 + x^24 + 1 (and its reciprocal) is the primitive trinomial behind
    the lags (24, 55): x^(2^55 - 1) = 1 mod p, and x^((2^55 - 1)/q) != 1 for each
    prime factor q of 2^55 - 1 (found here by trial division), so the low bits
    of a seeded stream have the full period 2^55 - 1."""
    p, deg = (1 << 55) | (1 << 31) | 1, 55
    order = 2**55 - 1
    assert _gf2_xpow(order, p, deg) == 1
    n, q, factors = order, 2, set()
    while q * q <= n:
        while n % q == 0:
            factors.add(q)
            n //= q
        q += 1
    if n > 1:
        factors.add(n)
    assert len(factors) >= 2
    for f in factors:
        assert _gf2_xpow(order // f, p, deg) != 1, f


def test_parisi_rapuano_uniformity():
    """10^6 outputs: odd fraction and the top-byte histogram of a uniform
    32-bit generator (5 sigma / chi-square with 255 degrees of freedom)."""
    out = oracle.pr_outputs(31337, 10**6)
    n = out.size
    assert abs((out & 1).mean() - 0.5) < 5 * 0.5 / math.sqrt(n)
    h = np.bincount(out >> 24, minlength=256)
    e = n / 256
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 255 + 5 * math.sqrt(2 * 255)


@pytest.mark.parametrize("beta", [1 / 1.1, 1 / 0.7, 1 / 0.9, 1 / 0.5, 1 / 1.5, 0.2, 0.05, 3.0])
def test_thresholds_high_precision(beta):
    pytest.importorskip("mpmath")
    assert list(oracle.thresholds(beta)) == _thr_mp(beta)


def test_thresholds_golden_and_limits():
    with open(os.path.join(GOLDEN, "thresholds.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for T, a, b, c in rows:
        assert list(oracle.thresholds(1.0 / float(T)))[1:] == [int(a), int(b), int(c)]
    assert list(oracle.thresholds(math.inf)) == [0, 0, 0, 0]
    t = oracle.thresholds(1e-12)          # beta -> 0+: every move accepted
    assert all(int(x) == 2**32 - 1 for x in t[1:])


# --------------------------------------------------------------------------
# Stencil logic: brute force over all 2^13 local configurations (Sec. 4)

def _paper_mask_decision(u, d, thr):
    """The paper's flip mask on one bit, read with sum = number of SATISFIED bonds
    (6 - u); cond_k = -(R < EXPk).  Returns True when the bit would flip."""
    sat = 6 - u
    s2, s1, s0 = (sat >> 2) & 1, (sat >> 1) & 1, sat & 1
    c12, c8, c4 = int(d < thr[3]), int(d < thr[2]), int(d < thr[1])
    mask = c12 | (1 - s2) | ((s2 & (s2 ^ s1)) & (c8 | (c4 & (1 - s0))))
    return bool(mask)


def test_stencil_exhaustive_energy_change():
    thr = oracle.thresholds(1 / 1.1)
    probes = sorted({0, 1, int(thr[3]) - 1, int(thr[3]), int(thr[2]) - 1, int(thr[2]),
                     int(thr[1]) - 1, int(thr[1]), 2**31, 2**32 - 1})
    seen_u = set()
    for code in range(1 << 13):
        bits = [(code >> k) & 1 for k in range(13)]
        s = 1 - 2 * bits[0]
        nb = [1 - 2 * b for b in bits[1:7]]
        J = [1 - 2 * b for b in bits[7:13]]
        u = oracle.unsatisfied(s, nb, J)
        # Eq. (1) restricted to the stencil of the site, before and after the flip
        h_before = -sum(J[k] * s * nb[k] for k in range(6))
        h_after = -sum(J[k] * (-s) * nb[k] for k in range(6))
        dE = h_after - h_before
        assert dE == 12 - 4 * u
        assert dE in (-12, -8, -4, 0, 4, 8, 12)            # Sec. 4 list of dE
        seen_u.add(u)
        if code % 17 == 0:
            for d in probes:
                dec = oracle.accept(u, d, thr)
                assert dec == _paper_mask_decision(u, d, thr), (u, d)
                if dE <= 0:
                    assert dec                                  # P_flip = 1 for dE <= 0
    assert seen_u == set(range(7))


# --------------------------------------------------------------------------
# Energy: closed forms for special configurations (Eq. 1)

@pytest.mark.parametrize("L", [4, 6, 8])
def test_energy_closed_forms(L):
    o = OracleSim(L, 1, 2, 1.0, RNG_MINSTD)
    N = L ** 3
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    checker = np.where(((x + y + z) % 2) == 0, 1, -1).astype(np.int8)
    checker = np.ascontiguousarray(np.transpose(checker, (2, 1, 0))).reshape(-1)  # i = x + L y + L^2 z
    o.set_couplings(np.ones((3, N), np.int8))
    o.set_spins(np.ones(N, np.int8))
    assert o.energy() == -3 * N                 # ferromagnet ground state
    o.set_spins(checker)
    assert o.energy() == 3 * N                  # every bond frustrated
    o.set_couplings(-np.ones((3, N), np.int8))
    assert o.energy() == -3 * N                 # antiferromagnet ground state
    # one coupling direction flipped: the x bonds change sign only
    J = np.ones((3, N), np.int8)
    J[0] = -1
    o.set_couplings(J)
    o.set_spins(np.ones(N, np.int8))
    assert o.energy() == -3 * N + 2 * N


@pytest.mark.parametrize("L", [4, 10])
def test_energy_symmetries(L):
    o = OracleSim(L, 11, 12, 1.0, RNG_MT19937)
    E = o.energy()
    N = L ** 3
    assert (E - 3 * N) % 2 == 0 and -3 * N <= E <= 3 * N
    s = o.spins()
    o.set_spins(-s)
    assert o.energy() == E                      # global spin flip
    o.close()


# --------------------------------------------------------------------------
# Dynamics invariants

@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L,beta", [(4, 0.3), (6, 1 / 1.1), (8, math.inf), (10, 1 / 0.7), (16, 1 / 1.1)])
def test_tracked_energy_equals_scratch(L, beta, kind):
    o = OracleSim(L, 3, 4, beta, kind)
    for _ in range(12):
        o.sweep(1)
        assert o.tracked_energy() == o.energy()


@pytest.mark.parametrize("kind", KINDS)
def test_zero_temperature_energy_nonincreasing(kind):
    o = OracleSim(16, 5, 6, math.inf, kind)
    E = [o.energy()]
    for _ in range(40):
        o.sweep(1)
        E.append(o.energy())
    assert all(b <= a for a, b in zip(E, E[1:]))
    assert E[-1] < E[0]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L", [8, 10])
def test_gauge_transform_maps_trajectory(L, kind):
    """sigma_i -> g_i sigma_i, J_ik -> g_i J_ik g_k leaves every u unchanged, and
    the draws do not depend on spin values, so the mapped trajectory is exact."""
    N = L ** 3
    rng = np.random.default_rng(2024 + L)
    g = rng.choice(np.array([-1, 1], np.int8), size=N)
    a = OracleSim(L, 21, 22, 1 / 1.1, kind)
    b = OracleSim(L, 21, 22, 1 / 1.1, kind)
    J = a.couplings()
    gg = g.reshape(L, L, L)                     # [z][y][x]
    Jp = np.empty_like(J)
    Jp[0] = (gg * J[0].reshape(L, L, L) * np.roll(gg, -1, axis=2)).reshape(-1)
    Jp[1] = (gg * J[1].reshape(L, L, L) * np.roll(gg, -1, axis=1)).reshape(-1)
    Jp[2] = (gg * J[2].reshape(L, L, L) * np.roll(gg, -1, axis=0)).reshape(-1)
    b.set_couplings(Jp)
    b.set_spins(g * a.spins())
    assert a.energy() == b.energy()
    for _ in range(15):
        a.sweep(1)
        b.sweep(1)
        assert np.array_equal(b.spins(), g * a.spins())
        assert a.energy() == b.energy() == b.tracked_energy()


def test_thread_count_does_not_change_result():
    a = OracleSim(64, 7, 8, 1 / 1.1, RNG_MT19937)     # 8 streams
    b = OracleSim(64, 7, 8, 1 / 1.1, RNG_MT19937)
    a.sweep(3, threads=1)
    b.sweep(3, threads=4)
    assert a.hash() == b.hash()
    assert np.array_equal(a.spins(), b.spins())
    assert a.tracked_energy() == b.tracked_energy()


# --------------------------------------------------------------------------
# Acceptance law: frequencies per u against min(1, exp(-beta dE)) (Sec. 4)

@pytest.mark.parametrize("kind,seed", [(RNG_MT19937, 99), (RNG_MINSTD, 12345), (RNG_PR, 4242)])
def test_acceptance_frequency_1e8(kind, seed):
    beta = 1 / 1.1
    n = 10**8
    acc = oracle.acceptance_trial(kind, seed, beta, n)
    for u in range(3):
        p = math.exp(-beta * (12 - 4 * u))
        sigma = math.sqrt(p * (1 - p) / n)
        assert abs(acc[u] / n - p) < 5 * sigma, (u, acc[u] / n, p)


@pytest.mark.parametrize("kind", KINDS)
def test_acceptance_frequency_in_sweeps(kind):
    beta = 0.3
    o = OracleSim(32, 31, 32, beta, kind)
    o.sweep(150)
    att, acc = o.move_counts()
    for u in range(7):
        if att[u] < 2000:
            continue
        p = min(1.0, math.exp(-beta * (12 - 4 * u)))
        if p == 1.0:
            assert acc[u] == att[u]
            continue
        sigma = math.sqrt(p * (1 - p) / att[u])
        assert abs(acc[u] / att[u] - p) < 5 * sigma, (u, acc[u] / att[u], p)


# --------------------------------------------------------------------------
# Equilibrium: high-temperature closed form E/N = -3 tanh(beta) (Eq. 3 with Eq. 1)

@pytest.mark.parametrize("kind", KINDS)
def test_equilibrium_energy_T5(kind):
    beta = 0.2
    o = OracleSim(32, 41, 42, beta, kind)
    o.sweep(200)
    es = []
    for _ in range(1000):
        o.sweep(1)
        es.append(o.tracked_energy() / o.N)
    assert o.tracked_energy() == o.energy()
    assert abs(np.mean(es) + 3 * math.tanh(beta)) < 2e-3


# --------------------------------------------------------------------------
# Measures, partition and arguments

def test_overlap_and_hash_properties():
    L = 8
    a = OracleSim(L, 1, 2, 1.0, RNG_MINSTD)
    b = OracleSim(L, 1, 3, 1.0, RNG_MINSTD)
    N = L ** 3
    assert a.overlap(a) == N
    s = a.spins()
    b.set_spins(-s)
    assert a.overlap(b) == -N
    h_pos = a.hash() ^ b.hash()                # Zobrist: H(s) ^ H(-s) = H(all +1)
    b.set_spins(np.ones(N, np.int8))
    assert b.hash() == h_pos
    b.set_spins(-np.ones(N, np.int8))
    assert b.hash() == 0
    # one spin up: the hash is that site's key
    one = -np.ones(N, np.int8)
    one[37] = 1
    b.set_spins(one)
    assert b.hash() == oracle.splitmix64(0xA54FF53A5F1D36F1, 37)


def test_stream_partition_and_draw_counts():
    table = {4: (16, 1), 16: (256, 1), 32: (1024, 1), 48: (768, 3), 64: (512, 8),
             96: (342, 27), 128: (256, 64), 192: (171, 216), 256: (128, 512),
             512: (64, 4096), 1024: (128, 8192), 2048: (512, 8192)}
    for L, (R, S) in table.items():
        assert (oracle.rows_per_stream(L), oracle.num_streams(L)) == (R, S)
        assert (S - 1) * R < L * L <= S * R
    o = OracleSim(96, 1, 2, 1.0, RNG_MT19937)
    o.sweep(2)
    assert o.draws_done(0) == 2 * 342 * 96
    assert o.draws_done(26) == 2 * (96 * 96 - 26 * 342) * 96


def test_coupling_and_spin_balance():
    o = OracleSim(32, 123, 456, 1.0, RNG_MINSTD)
    J = o.couplings()
    s = o.spins()
    n = J.size
    assert abs((J == -1).mean() - 0.5) < 5 * math.sqrt(0.25 / n)   # Eq. (2): p = 1/2
    assert abs((s == -1).mean() - 0.5) < 5 * math.sqrt(0.25 / s.size)


@pytest.mark.parametrize("args", [(5, 0.5, 0), (2, 0.5, 0), (8, 0.0, 0), (8, -1.0, 0),
                                  (8, float("nan"), 0), (8, 0.5, 3), (2050, 0.5, 0)])
def test_invalid_arguments_rejected(args):
    L, beta, kind = args
    with pytest.raises(ValueError):
        OracleSim(L, 1, 2, beta, kind)


# ------------------------------------------------- one site at a time ---

@pytest.mark.parametrize("kind", [RNG_MINSTD, RNG_MT19937, RNG_PR])
def test_per_site_initial_state_and_stream_words(kind):
    """The per-site helpers draw the same initial state and stream seeds as the
    simulator (Eq. (2)): every spin and coupling of an L = 10 lattice, and the
    first draws of every stream of an L = 66 lattice (8 streams)."""
    L = 10
    o = OracleSim(L, 7, 8, 1.0, kind)
    s, J = o.spins(), o.couplings().reshape(3, -1)
    for i in range(L ** 3):
        assert s[i] == oracle.initial_spin(8, i)
        for d in range(3):
            assert J[d, i] == oracle.initial_coupling(7, i, d)
    o = OracleSim(66, 7, 8, 1.0, kind)
    for t in range(oracle.num_streams(66)):
        assert np.array_equal(o.peek_draws(t, 300), oracle.stream_draws(kind, oracle.stream_word(8, t), 300))


@pytest.mark.parametrize("kind", [RNG_MINSTD, RNG_MT19937, RNG_PR])
@pytest.mark.parametrize("L", [8, 66])
def test_sampled_first_sweep_matches_simulator(L, kind):
    """SampledFirstSweep (the check used at L = 2048, where OracleSim does not
    fit in memory) against OracleSim after one sweep: every site at L = 8 (one
    stream), and at L = 66 (8 streams of 545 rows, the last one 541) the sites
    of the rows at every stream boundary plus 2000 random sites."""
    beta = 1 / 0.8
    o = OracleSim(L, 3, 4, beta, kind)
    o.sweep(1)
    sp = o.spins()
    smp = oracle.SampledFirstSweep(L, 3, 4, beta, kind)
    if L <= 8:
        sites = [(x, y, z) for z in range(L) for y in range(L) for x in range(L)]
    else:
        R = oracle.rows_per_stream(L)
        rows = sorted({r for t in range(oracle.num_streams(L)) for r in (t * R - 1, t * R) if 0 <= r < L * L})
        sites = [(x, r % L, r // L) for r in rows for x in range(L)]
        rng = np.random.default_rng(5)
        sites += [tuple(int(v) for v in rng.integers(0, L, 3)) for _ in range(2000)]
    flips = 0
    for x, y, z in sites:
        got = smp.after(x, y, z)
        assert got == sp[x + L * y + L * L * z], (x, y, z)
        flips += got != smp.initial(x, y, z)
    assert flips > len(sites) // 10          # the sweep did change many of them
