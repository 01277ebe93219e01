"""GPU path (through the C-ABI) against the CPU oracle.  Tolerance is zero
everywhere: the Metropolis trajectory is exact integer arithmetic, so spins,
energies and hashes must agree bit for bit.

Sizes span one and several word groups per warp, ragged rows (L/2 not a multiple
of the word width), 32- and 64-bit words, one and many RNG streams, and the
degenerate temperatures beta = inf and beta -> 0."""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleSim

pytestmark = pytest.mark.gpu

K_STREAMS = 0x3C6EF372FE94F82B
KINDS = ["minstd", "mt19937", "parisi_rapuano"]


def raw_outputs(kind, v, n):
    """The oracle's raw outputs of a stream with seed word v, as the kernels
    compare them: MT19937 and Parisi-Rapuano as is, MINSTD doubled."""
    if kind == "mt19937":
        return oracle.mt19937_outputs(v & 0xFFFFFFFF, n)
    if kind == "parisi_rapuano":
        return oracle.pr_outputs(v, n)
    return (oracle.minstd_outputs(1 + v % (2**31 - 2), n) << 1).astype(np.uint32)


@pytest.fixture(scope="module")
def isg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_0127_gb300 import build
    build.build()
    import paper_1411_0127_gb300 as m
    return m


def pair(isg, L, kind, beta, seed_J=1, seed_spin=2):
    return (isg.Sim(L, seed_J, seed_spin, beta, kind),
            OracleSim(L, seed_J, seed_spin, beta, isg.RNG_KINDS[kind]))


# ------------------------------------------------------------- bit logic ---

def test_stencil_logic_exhaustive(isg):
    """All 2^13 stencils x draws at and around every threshold: the kernel's
    bit-sliced adder and flip mask against the oracle's bond-by-bond rule."""
    for beta in (1 / 1.1, 1 / 0.7, 0.3, math.inf):
        thr = oracle.thresholds(beta)
        probes = sorted({0, 1, 2**31, 2**32 - 1} |
                        {int(t) + dd for t in thr[1:] for dd in (-1, 0, 1) if 0 <= int(t) + dd < 2**32})
        codes = np.repeat(np.arange(1 << 13, dtype=np.uint16), len(probes))
        draws = np.tile(np.array(probes, dtype=np.uint32), 1 << 13)
        flip, u = isg.stencil_decisions(codes, draws, thr[1:])
        assert (u != 0xFF).all(), "32- and 64-bit word logic disagree"
        for j in range(0, codes.size, 7):       # every 7th pair through the oracle (ctypes is slow)
            c = int(codes[j])
            s = 1 - 2 * (c & 1)
            nb = [1 - 2 * ((c >> (1 + k)) & 1) for k in range(6)]
            Jk = [1 - 2 * ((c >> (7 + k)) & 1) for k in range(6)]
            uo = oracle.unsatisfied(s, nb, Jk)
            assert u[j] == uo, (c, u[j], uo)
            assert bool(flip[j]) == oracle.accept(uo, int(draws[j]), thr), (c, int(draws[j]))


# ---------------------------------------------------------------- streams ---

@pytest.mark.parametrize("kind", KINDS)
def test_stream_draws(isg, kind):
    g, o = pair(isg, 96, kind, 1.0)                 # 27 streams
    for t in (0, 1, 13, 26):
        assert np.array_equal(g.peek_draws(t, 5000), o.peek_draws(t, 5000)), t
    # independently of the oracle's stream set-up: the library generators
    v = oracle.splitmix64(2 ^ K_STREAMS, 5)
    assert np.array_equal(g.peek_draws(5, 3000), raw_outputs(kind, v, 3000))
    # after sweeps the streams continue where the oracle's do
    g.sweep(2)
    o.sweep(2)
    for t in (0, 26):
        assert np.array_equal(g.peek_draws(t, 777), o.peek_draws(t, 777))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [1000, 4096, 20001])
def test_generator_benchmark_counts(isg, kind, n):
    """The device-API benchmark (odd outputs) against the oracle's generators,
    seeded like lattice streams: counts must be equal."""
    seed, streams = 77, 5
    odd, ms = isg.rng_count_odd(kind, seed, streams, n)
    ref = 0
    for t in range(streams):
        v = oracle.splitmix64(seed ^ K_STREAMS, t)
        out = (oracle.minstd_outputs(1 + v % (2**31 - 2), n) if kind == "minstd"   # the state x itself
               else raw_outputs(kind, v, n))
        ref += int((out & 1).sum())
    assert odd == ref
    assert ms >= 0.0


def test_integer_rate_microbenchmark(isg):
    """The measured integer rates are positive and below the issue limit
    (SMs x 128 lanes x the maximum clock, with 10 % of slack for timing)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    limit = sms * 128 * 2.1e9 * 1.1
    for mode in (0, 1, 2):
        r = isg.int_rate(mode)
        assert 0 < r < limit, (mode, r)


# ------------------------------------------------------------------- init ---

@pytest.mark.parametrize("L", [4, 6, 16, 32, 48, 96, 130])
def test_initial_state(isg, L):
    g, o = pair(isg, L, "minstd", 1.0, seed_J=123, seed_spin=456)
    assert np.array_equal(g.read_spins(), o.spins())
    assert np.array_equal(g.read_couplings(), o.couplings())
    assert g.energy() == o.energy() == g.tracked_energy()
    assert g.hash() == o.hash()


# ------------------------------------------------------------- trajectory ---

RAGGED = [4, 6, 8, 10, 14, 18, 34, 46, 62, 66, 94, 98, 130, 192]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L", RAGGED)
def test_trajectory_ragged_sizes(isg, L, kind):
    g, o = pair(isg, L, kind, 1 / 1.1, seed_J=L, seed_spin=3 * L + 1)
    sweeps = 6 if L <= 98 else 3
    for _ in range(sweeps):
        g.sweep(1)
        o.sweep(1, threads=8)
        assert np.array_equal(g.read_spins(), o.spins()), (L, kind)
        assert g.tracked_energy() == o.tracked_energy()
    assert g.energy() == o.energy()
    assert g.hash() == o.hash()


@pytest.mark.parametrize("beta", [math.inf, 1e-9, 0.05, 3.0])
def test_trajectory_extreme_temperatures(isg, beta):
    for kind in KINDS:
        g, o = pair(isg, 20, kind, beta)
        g.sweep(5)
        o.sweep(5)
        assert np.array_equal(g.read_spins(), o.spins())
        assert g.tracked_energy() == o.tracked_energy() == g.energy()


def test_small_workload_every_sweep(isg):
    """L = 32, seeds 1/2, T = 1.1, MINSTD, 1000 sweeps: integer energy and spin
    hash compared after every sweep."""
    from paper_1411_0127_gb300 import workloads
    w = workloads.SMALL
    g, o = pair(isg, w.L, w.kind, w.beta, w.seed_J, w.seed_spin)
    for k in range(w.sweeps):
        g.sweep(1)
        o.sweep(1)
        assert g.tracked_energy() == o.tracked_energy(), k
        assert g.hash() == o.hash(), k
    assert g.energy() == o.energy()
    assert np.array_equal(g.read_spins(), o.spins())


@pytest.mark.parametrize("kind,kmax", [
    pytest.param("minstd", 13, marks=pytest.mark.slow),
    pytest.param("mt19937", 13, marks=pytest.mark.slow),
    ("parisi_rapuano", 10),
])
def test_medium_workload_powers_of_two(isg, kind, kmax):
    """L = 256, T = 0.7: energy and hash at sweeps 2^k, k = 0..kmax.  MINSTD
    and MT19937 run the workload's stated length (10^4 sweeps, measured at
    every 2^k up to 2^13 = 8192); the third generator to 2^10."""
    g, o = pair(isg, 256, kind, 1 / 0.7)
    done = 0
    for k in range(kmax + 1):
        n = 2**k - done
        g.sweep(n)
        o.sweep(n, threads=16)
        done = 2**k
        assert g.tracked_energy() == o.tracked_energy(), k
        assert g.hash() == o.hash(), k
    assert g.energy() == o.energy()
    assert np.array_equal(g.read_spins(), o.spins())


@pytest.mark.slow
def test_large_workload_powers_of_two(isg):
    """L = 1024, MT19937, T = 0.9 -- the benchmarked configuration, launched as
    the benchmark launches it: tracked energy and hash against the oracle at
    sweeps 1, 2, 4, ..., 32, the energy from scratch and all 2^30 spins at the
    end."""
    from paper_1411_0127_gb300 import workloads
    w = workloads.LARGE
    g, o = pair(isg, w.L, w.kind, w.beta, w.seed_J, w.seed_spin)
    assert g.hash() == o.hash()
    done = 0
    for k in range(6):
        n = 2**k - done
        g.sweep(n)
        o.sweep(n, threads=16)
        done = 2**k
        assert g.tracked_energy() == o.tracked_energy(), k
        assert g.hash() == o.hash(), k
    assert g.energy() == o.energy()
    assert np.array_equal(g.read_spins(), o.spins())


@pytest.mark.parametrize("kind", KINDS)
def test_maximum_size_sampled(isg, kind):
    """L = 2048, the largest lattice the ABI accepts: 8.6e9 spins, 4 GiB of bit
    planes on the device, 34 GB as OracleSim's int8 arrays (too large to hold).
    The initial spins and the spins after one sweep at sampled sites (rows at
    stream boundaries and the lattice's last row, x at both ends and at word
    boundaries, and random sites) are recomputed one by one by the oracle
    (SampledFirstSweep); the energy bookkeeping is checked as a property that
    holds at any size (tracked = from scratch)."""
    L, beta = 2048, 1 / 0.9
    g = isg.Sim(L, 1, 2, beta, kind)
    smp = oracle.SampledFirstSweep(L, 1, 2, beta, isg.RNG_KINDS[kind])
    R, S = oracle.rows_per_stream(L), oracle.num_streams(L)
    sites = []
    for r in (0, R - 1, R, (S // 2) * R, (S - 1) * R - 1, (S - 1) * R, L * L - 1):
        for x in (0, 1, 2, 63, 64, 65, L // 2 - 1, L // 2, L - 2, L - 1):
            sites.append((x, r % L, r // L))
    rng = np.random.default_rng(11)
    sites += [tuple(int(v) for v in rng.integers(0, L, 3)) for _ in range(300)]

    def spin(bits, x, y, z):
        i = x + L * y + L * L * z
        return 1 if (int(bits[i >> 3]) >> (i & 7)) & 1 else -1

    smp.prefetch(sites)
    bits = g.read_spins_packed()
    for x, y, z in sites:
        assert spin(bits, x, y, z) == smp.initial(x, y, z), (x, y, z)
    g.sweep(1)
    g.read_spins_packed(out=bits)
    flips = 0
    for x, y, z in sites:
        want = smp.after(x, y, z)
        assert spin(bits, x, y, z) == want, (x, y, z)
        flips += want != smp.initial(x, y, z)
    assert flips > len(sites) // 10
    E = g.tracked_energy()
    assert E == g.energy()
    assert abs(E) <= 3 * L ** 3 and (E - 3 * L ** 3) % 2 == 0
    g.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L", [432, 512])
def test_throughput_form_lattices(isg, L, kind):
    """Lattices with at least 16 streams per SM (2456 and 4096 streams here) run
    the throughput form of the draw phase (one comparison per draw when no draw
    of a quad is below the second threshold); L = 432 has 32-bit words, L = 512
    64-bit words.  Three sweeps at T = 1.1 against the oracle, all spins."""
    g, o = pair(isg, L, kind, 1 / 1.1, seed_J=L + 1, seed_spin=L + 2)
    assert g.info()["streams"] >= 2432
    g.sweep(3)
    o.sweep(3, threads=16)
    assert g.tracked_energy() == o.tracked_energy()
    assert g.hash() == o.hash()
    assert np.array_equal(g.read_spins(), o.spins())


@pytest.mark.parametrize("kind", ["minstd", "mt19937"])
@pytest.mark.parametrize("L", [640, 704])
def test_multi_pass_launches(isg, L, kind):
    """MT19937 and MINSTD lattices with more streams than a launch has warps
    (L = 640: 7877 streams, 64-bit words; L = 704: 8125 streams, 32-bit words)
    run all passes
    of an isg_sweep call in persistent launches of up to 64 sweeps, each
    stream's pass starting once its neighbouring streams have finished the
    previous one (L = 432 and 512 keep one launch per pass; calls of fewer
    than 8 sweeps too).  65 sweeps in one call (two launches: 64 + 1), the same
    65 as one call per sweep, and the plain per-colour kernel reach the same
    configuration; ten sweeps in calls of 1 + 9 against the oracle, all spins;
    an exchange of ten sweeps (one of single passes, then nine in a multi-pass
    launch) continues the same trajectory."""
    a = isg.Sim(L, L + 3, L + 4, 1 / 0.9, kind)
    b = isg.Sim(L, L + 3, L + 4, 1 / 0.9, kind)
    c = isg.Sim(L, L + 3, L + 4, 1 / 0.9, kind)
    assert a.passes_per_launch() == 128
    assert isg.Sim(512, 1, 2, 1.0, kind).passes_per_launch() == 1
    assert isg.Sim(L, 1, 2, 1.0, "parisi_rapuano").passes_per_launch() == 1
    a.sweep(65)
    for _ in range(65):
        b.sweep(1)
    c.sweep_plain(65)
    assert a.hash() == b.hash() == c.hash()
    assert a.tracked_energy() == b.tracked_energy() == c.tracked_energy() == a.energy()
    for h in (a, b, c):
        h.close()
    g, o = pair(isg, L, kind, 1 / 1.1, seed_J=L + 5, seed_spin=L + 6)
    g.sweep(1)
    g.sweep(9)
    o.sweep(10, threads=16)
    assert g.tracked_energy() == o.tracked_energy()
    assert np.array_equal(g.read_spins(), o.spins())
    bits = g.read_spins_packed()
    E = np.zeros(1, dtype=np.int64)
    g.exchange_async(bits, None, 10, E)     # one sweep of single passes, then a multi-pass launch
    o.sweep(10, threads=16)
    import torch
    torch.cuda.synchronize()
    assert int(E[0]) == g.tracked_energy() == o.tracked_energy() == g.energy()
    assert g.hash() == o.hash()


def test_multi_pass_launches_maximum_size(isg):
    """L = 2048, the largest lattice (8192 streams of 512 rows: a stream's z
    neighbours are 4 streams away): 8 MT19937 sweeps in one multi-pass launch
    equal 8 calls of one sweep (one launch per colour pass), and the tracked
    energy equals the energy from scratch."""
    a = isg.Sim(2048, 1, 2, 1 / 0.9, "mt19937")
    assert a.passes_per_launch() == 128
    a.sweep(8)
    ha, Ea = a.hash(), a.tracked_energy()
    assert Ea == a.energy()
    a.close()
    b = isg.Sim(2048, 1, 2, 1 / 0.9, "mt19937")
    for _ in range(8):
        b.sweep(1)
    assert b.hash() == ha and b.tracked_energy() == Ea
    b.close()


def test_multi_pass_wait_gives_up_with_a_status(isg):
    """A multi-pass launch whose second pass waits for a pass that never comes
    (the isg_sweep_test_stall hook): its bounded waits run out, the rest of the
    launch is skipped, the next energy read reports ISG_ERR_TIMEOUT once, and the
    context stays usable."""
    g = isg.Sim(640, 1, 2, 1 / 0.9, "minstd")
    assert isg.lib().isg_sweep_test_stall(g.handle) == isg.ISG_OK
    g.sweep(8)
    with pytest.raises(isg.IsgError) as ei:
        g.tracked_energy()
    assert ei.value.code == isg.ISG_ERR_TIMEOUT
    g.tracked_energy()                       # reported once
    g.close()
    small = isg.Sim(64, 1, 2, 1 / 0.9, "minstd")
    assert isg.lib().isg_sweep_test_stall(small.handle) == isg.ISG_ERR_STATE
    h, o = pair(isg, 640, "mt19937", 1 / 0.9)
    h.sweep(8)
    o.sweep(8, threads=16)
    assert h.tracked_energy() == o.tracked_energy() == h.energy()


@pytest.mark.parametrize("L", [32, 50, 96, 130])
def test_segmented_minstd_streams(isg, L):
    """MINSTD lattices with few streams run every stream as several row-group
    segments started by jump-ahead, the end states going to a second buffer.
    L = 50 and 130 leave empty segments in the short last stream.  Sweeps
    against the oracle, stream states (peek) after every sweep, the plain
    kernel in between, and a checkpoint taken mid-run that resumes identically."""
    g, o = pair(isg, L, "minstd", 1 / 1.1, seed_J=L + 7, seed_spin=L + 8)
    for s in range(4):
        (g.sweep_plain if s == 2 else g.sweep)(1)
        o.sweep(1)
        assert np.array_equal(g.read_spins(), o.spins()), (L, s)
        assert g.tracked_energy() == o.tracked_energy() == g.energy()
        for t in {0, g.info()["streams"] - 1}:
            assert np.array_equal(g.peek_draws(t, 65), o.peek_draws(t, 65)), (L, s, t)
    c = isg.Sim.load(g.save())
    g.sweep(2)
    c.sweep(2)
    o.sweep(2)
    assert g.hash() == c.hash() == o.hash()


@pytest.mark.parametrize("L", [4, 10, 34, 64, 128, 130, 256])
def test_spin_io_formats(isg, L):
    """int8 and packed-bit spin I/O against the oracle: L = 64, 128 and 256 take
    the vector path of the int8 packer (L a multiple of twice the word width),
    the others the scalar path, with rows that start inside words and tails
    shorter than 16 or 32 sites."""
    g, o = pair(isg, L, "mt19937", 1 / 0.9, seed_J=L, seed_spin=L + 1)
    g.sweep(3)
    o.sweep(3)
    ref = o.spins()
    np.testing.assert_array_equal(g.read_spins(), ref)
    bits = g.read_spins_packed()
    np.testing.assert_array_equal(bits, np.packbits(ref == 1, bitorder="little"))
    # round trips through both formats, with another configuration
    rng = np.random.default_rng(L)
    s = np.where(rng.random(L**3) < 0.5, 1, -1).astype(np.int8)
    g.write_spins(s)
    np.testing.assert_array_equal(g.read_spins(), s)
    assert g.tracked_energy() == g.energy()
    s2 = -s
    g.write_spins_packed(np.packbits(s2 == 1, bitorder="little"))
    np.testing.assert_array_equal(g.read_spins(), s2)
    np.testing.assert_array_equal(g.read_spins_packed(), np.packbits(s2 == 1, bitorder="little"))
    assert g.tracked_energy() == g.energy()
    o.set_spins(s2)
    assert g.energy() == o.energy()
    # a rejected int8 array changes nothing
    bad = s.copy()
    bad[L**3 // 2] = 0
    with pytest.raises(isg.IsgError):
        g.write_spins(bad)
    np.testing.assert_array_equal(g.read_spins(), s2)
    # reading into a caller's buffer
    buf = np.zeros(L**3 + 5, dtype=np.int8)
    assert g.read_spins(out=buf) is buf
    np.testing.assert_array_equal(buf[:L**3], s2)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L", [10, 64])
def test_exchange_async(isg, L, kind):
    """isg_exchange_async against the oracle: a configuration in, sweeps, the
    configuration and the tracked energy out, enqueued with no synchronisation;
    then without an input; then a pipeline of nine exchanges over three handles
    on three streams equals the same exchanges made one after another."""
    torch = pytest.importorskip("torch")
    N, nb = L ** 3, (L ** 3 + 7) // 8

    def pinned(n, dtype):
        return torch.zeros(n, dtype=dtype).pin_memory().numpy()

    def unpack(bits):
        return (np.unpackbits(bits, bitorder="little")[:N].astype(np.int8) * 2 - 1).astype(np.int8)

    g, o = pair(isg, L, kind, 1 / 0.9, seed_J=3, seed_spin=4)
    rng = np.random.default_rng(L)
    s = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int8)
    b_in, b_out, E = pinned(nb, torch.uint8), pinned(nb, torch.uint8), pinned(1, torch.int64)
    b_in[:] = np.packbits(s == 1, bitorder="little")
    st = torch.cuda.Stream()
    g.exchange_async(b_in, b_out, 3, E, st)
    st.synchronize()
    o.set_spins(s)
    o.sweep(3)
    assert np.array_equal(unpack(b_out), o.spins())
    assert int(E[0]) == o.energy() == g.energy() == g.tracked_energy()
    g.exchange_async(None, b_out, 2, E, st)
    st.synchronize()
    o.sweep(2)
    assert np.array_equal(unpack(b_out), o.spins())
    assert int(E[0]) == o.energy()
    # a configuration in with no sweep: the bookkeeping restarts by a separate popcount pass
    b_in[:] = np.packbits(-s == 1, bitorder="little")
    g.exchange_async(b_in, b_out, 0, E, st)
    st.synchronize()
    o.set_spins((-s).astype(np.int8))
    assert np.array_equal(unpack(b_out), o.spins())
    assert int(E[0]) == o.energy() == g.energy() == g.tracked_energy()
    # and with one sweep: the first colour pass counts the bonds before its flips
    g.exchange_async(b_in, b_out, 1, E, st)
    st.synchronize()
    o.sweep(1)
    assert np.array_equal(unpack(b_out), o.spins())
    assert int(E[0]) == o.energy() == g.energy() == g.tracked_energy()

    def run(pipelined):
        hs = [isg.Sim(L, 5 + j, 6 + j, 1 / 0.8, kind) for j in range(3)]
        streams = [torch.cuda.Stream() for _ in range(3)] if pipelined else [torch.cuda.current_stream()] * 3
        ins = [pinned(nb, torch.uint8) for _ in range(9)]
        outs = [pinned(nb, torch.uint8) for _ in range(9)]
        Es = [pinned(1, torch.int64) for _ in range(9)]
        r = np.random.default_rng(99)
        for k in range(9):
            ins[k][:] = r.integers(0, 256, nb, dtype=np.uint8)
        for k in range(9):
            hs[k % 3].exchange_async(ins[k] if k % 2 == 0 else None, outs[k], 1 + k % 2, Es[k], streams[k % 3])
            if not pipelined:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        res = [(o_.copy(), int(e_[0])) for o_, e_ in zip(outs, Es)]
        for h in hs:
            assert h.tracked_energy() == h.energy()
            h.close()
        return res

    a, b = run(True), run(False)
    for (oa, ea), (ob, eb) in zip(a, b):
        assert np.array_equal(oa, ob) and ea == eb


def test_empty_work_and_short_buffers(isg):
    """Zero sweeps change nothing anywhere (lattice, batch, ensemble, exchange);
    buffers shorter than the configuration are refused before any device work."""
    import ctypes
    torch = pytest.importorskip("torch")
    g = isg.Sim(34, 1, 2, 1 / 0.9, "mt19937")
    h0, E0 = g.hash(), g.tracked_energy()
    g.sweep(0)
    assert g.hash() == h0 and g.tracked_energy() == E0 and g.sweeps_done() == 0
    E = torch.zeros(1, dtype=torch.int64).pin_memory().numpy()
    g.exchange_async(None, None, 0, E)
    torch.cuda.synchronize()
    assert int(E[0]) == E0 and g.hash() == h0
    nb = (34 ** 3 + 7) // 8
    short = np.zeros(nb - 1, dtype=np.uint8)
    lib = isg.lib()
    assert lib.isg_exchange_async(g._h, short.ctypes.data, None, short.size, 1, None, None) == isg.ISG_ERR_ARG
    assert lib.isg_exchange_async(g._h, None, short.ctypes.data, short.size, 1, None, None) == isg.ISG_ERR_ARG
    assert lib.isg_read_spins_packed(g._h, short.ctypes.data, short.size, None) == isg.ISG_ERR_ARG
    assert lib.isg_sweep(g._h, -1, None) == isg.ISG_ERR_ARG
    assert g.hash() == h0 and g.sweeps_done() == 0
    g.close()
    b = isg.Batch([16, 20], [1, 2], [3, 4, 5, 6], [1.0, 1.2], "minstd")
    Eb, Hb = b.tracked()
    b.run(0)
    Eb2, Hb2 = b.tracked()
    assert np.array_equal(Eb, Eb2) and np.array_equal(Hb, Hb2)
    b.close()
    from paper_1411_0127_gb300 import workloads
    J, S = workloads.amsc_seeds(16)
    m = isg.Amsc(16, J, S, 7, 1 / 0.9, "minstd")
    Em = m.energies()
    m.sweep(0)
    assert np.array_equal(m.energies(), Em)
    m.close()


# ------------------------------------------------------------- invariants ---

@pytest.mark.parametrize("kind", KINDS)
def test_tracked_energy_long_run(isg, kind):
    g = isg.Sim(128, 9, 10, 1 / 0.9, kind)
    for _ in range(5):
        g.sweep(200)
        assert g.tracked_energy() == g.energy()


def test_plain_and_default_sweep_agree(isg):
    a = isg.Sim(64, 5, 6, 1 / 1.1, "mt19937")
    b = isg.Sim(64, 5, 6, 1 / 1.1, "mt19937")
    a.sweep(7)
    b.sweep_plain(7)
    assert a.hash() == b.hash() and a.tracked_energy() == b.tracked_energy()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L", [6, 48, 98, 256])
def test_fast_and_plain_kernels_interleaved(isg, L, kind):
    """The two flip kernels share the stream-state format: alternating them on
    one handle follows the oracle's trajectory."""
    g, o = pair(isg, L, kind, 1 / 0.9, seed_J=7, seed_spin=8)
    for k in range(6):
        (g.sweep if k % 2 == 0 else g.sweep_plain)(1)
        o.sweep(1, threads=8)
        assert g.tracked_energy() == o.tracked_energy(), k
    assert np.array_equal(g.read_spins(), o.spins())


def test_gauge_transform_on_gpu(isg):
    L = 24
    rng = np.random.default_rng(5)
    g = rng.choice(np.array([-1, 1], np.int8), size=L**3)
    a = isg.Sim(L, 21, 22, 1 / 1.1, "mt19937")
    b = isg.Sim(L, 21, 22, 1 / 1.1, "mt19937")
    J = a.read_couplings()
    gg = g.reshape(L, L, L)
    Jp = np.stack([(gg * J[0].reshape(L, L, L) * np.roll(gg, -1, axis=2)).reshape(-1),
                   (gg * J[1].reshape(L, L, L) * np.roll(gg, -1, axis=1)).reshape(-1),
                   (gg * J[2].reshape(L, L, L) * np.roll(gg, -1, axis=0)).reshape(-1)])
    b.write_couplings(Jp)
    b.write_spins(g * a.read_spins())
    for _ in range(10):
        a.sweep(1)
        b.sweep(1)
        assert np.array_equal(b.read_spins(), g * a.read_spins())
        assert a.tracked_energy() == b.tracked_energy() == b.energy()


def test_special_configurations_energy(isg):
    L = 10
    N = L**3
    g = isg.Sim(L, 1, 2, 1.0, "minstd")
    g.write_couplings(np.ones((3, N), np.int8))
    g.write_spins(np.ones(N, np.int8))
    assert g.energy() == -3 * N
    x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    checker = np.ascontiguousarray(np.transpose(np.where((x + y + z) % 2 == 0, 1, -1), (2, 1, 0))).reshape(-1)
    g.write_spins(checker.astype(np.int8))
    assert g.energy() == 3 * N
    with pytest.raises(isg.IsgError):
        g.write_spins(np.zeros(N, np.int8))
    assert g.energy() == 3 * N


def test_overlap(isg):
    a = isg.Sim(40, 77, 1, 1 / 0.9, "minstd")
    b = isg.Sim(40, 77, 2, 1 / 0.9, "minstd")
    oa = OracleSim(40, 77, 1, 1 / 0.9, 0)
    ob = OracleSim(40, 77, 2, 1 / 0.9, 0)
    for _ in range(3):
        a.sweep(4)
        b.sweep(4)
        oa.sweep(4)
        ob.sweep(4)
        assert a.overlap(b) == oa.overlap(ob)
    assert a.overlap(a) == 40**3
    c = isg.Sim(40, 78, 1, 1.0, "minstd")
    with pytest.raises(isg.IsgError) as ei:
        a.overlap(c)
    assert ei.value.code == isg.ISG_ERR_MISMATCH


# --------------------------------------------------------------- plumbing ---

@pytest.mark.parametrize("kind", KINDS)
def test_checkpoint_resume(isg, kind):
    a = isg.Sim(48, 3, 4, 1 / 0.9, kind)
    a.sweep(5)
    blob = a.save()
    a.sweep(7)
    b = isg.Sim.load(blob)
    assert b.sweeps_done() == 5
    b.sweep(7)
    assert a.hash() == b.hash()
    assert a.tracked_energy() == b.tracked_energy() == b.energy()
    assert np.array_equal(a.read_spins(), b.read_spins())
    with pytest.raises(isg.IsgError):
        isg.Sim.load(blob[:100])


def test_torch_allocator_and_streams(isg):
    import torch
    isg.use_torch_allocator()
    try:
        s = torch.cuda.Stream()
        a = isg.Sim(64, 1, 2, 1 / 1.1, "mt19937")
        a.sweep(3, stream=s)
        s.synchronize()
        o = OracleSim(64, 1, 2, 1 / 1.1, 1)
        o.sweep(3)
        assert a.hash(stream=s) == o.hash()
        a.close()
    finally:
        isg.use_default_allocator()
