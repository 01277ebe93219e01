"""Batched persistent engine against lone lattices and the CPU oracle.  Every
replica of a batch must follow, bit for bit, the trajectory of a lone handle
with the same seeds (and so the oracle's): tolerance zero."""
import numpy as np
import pytest

import oracle
from oracle import OracleSim

pytestmark = pytest.mark.gpu

SIZES = (16, 32, 48, 64, 96, 128, 192)


@pytest.fixture(scope="module")
def isg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_0127_gb300 import build
    build.build()
    import paper_1411_0127_gb300 as m
    return m


def mixed(n_per_size=1, temps=(0.7, 1.1)):
    L, J, S, B = [], [], [], []
    s = 0
    for size in SIZES:
        for T in temps:
            for _ in range(n_per_size):
                L.append(size)
                J.append(500 + s)
                S += [2 * s + 11, 2 * s + 12]
                B.append(1.0 / T)
                s += 1
    return L, J, S, B


@pytest.mark.parametrize("kind", ["mt19937", "minstd", "parisi_rapuano"])
def test_batch_matches_oracle(isg, kind):
    L, J, S, B = mixed()
    b = isg.Batch(L, J, S, B, kind)
    b.run(8, group_sweeps=3)              # two graph replays of 3 sweeps, then 2 more
    E, Q = b.measure()
    Et, H = b.tracked()
    assert np.array_equal(E, Et)
    k = isg.RNG_KINDS[kind]
    for s in range(len(L)):
        o = [OracleSim(L[s], J[s], S[2 * s + j], B[s], k) for j in range(2)]
        for j in range(2):
            o[j].sweep(8, threads=8)
            assert E[2 * s + j] == o[j].tracked_energy(), (s, j, L[s])
            assert int(H[2 * s + j]) == o[j].hash(), (s, j)
        assert Q[s] == o[0].overlap(o[1]), s
        if L[s] <= 64:
            assert np.array_equal(b.member(2 * s).read_spins(), o[0].spins())


def test_batch_member_equals_lone_handle(isg):
    L, J, S, B = mixed(n_per_size=2, temps=(0.9,))
    b = isg.Batch(L, J, S, B, "mt19937")
    lone = [isg.Sim(L[r // 2], J[r // 2], S[r], B[r // 2], "mt19937") for r in range(2 * len(L))]
    for g in (5, 64):                     # group shorter and longer than the run
        b.run(5, group_sweeps=g)
        for m in lone:
            m.sweep(5)
        E, H = b.tracked()
        for r, m in enumerate(lone):
            assert H[r] == m.hash() and E[r] == m.tracked_energy(), (g, r, L[r // 2])
    assert b.info()["samples"] == len(L)


@pytest.mark.parametrize("config", [(0, 32, 1, 1), (4, 4, 0, 2), (5, 4, 0, 1)])
def test_full_batch_workload_sampled(isg, config):
    """The 512-sample workload in one graph-replayed persistent launch of 64
    sweeps, with the default bundle configuration and with both pass engines
    (the per-pass form is the one the autotuner picks for MT19937, the
    benchmark's configuration); energies and
    overlaps of one sample per lattice size checked against the oracle, the
    energy bookkeeping of every replica checked against its energy from
    scratch."""
    from paper_1411_0127_gb300 import workloads
    samples = workloads.batch_samples()
    L = [x.L for x in samples]
    b = isg.Batch(L, [x.seed_J for x in samples], [v for x in samples for v in x.seed_spin],
                  [1.0 / x.T for x in samples], "mt19937")
    b.set_config(*config)
    info = b.info()
    assert info["attempts_per_sweep"] == 2 * sum(v ** 3 for v in L)
    b.run(64, group_sweeps=64)
    E, Q = b.measure()
    Et, H = b.tracked()
    assert np.array_equal(E, Et)
    N = np.array([v ** 3 for v in L])
    assert (np.abs(Q) <= N).all()
    picked = {}
    for s, v in enumerate(L):
        picked.setdefault(v, s)
    for v, s in sorted(picked.items()):
        x = samples[s]
        for j in range(2):
            o = OracleSim(x.L, x.seed_J, x.seed_spin[j], 1.0 / x.T, oracle.RNG_MT19937)
            o.sweep(64, threads=16)
            assert E[2 * s + j] == o.tracked_energy(), (v, s, j)
            assert int(H[2 * s + j]) == o.hash(), (v, s, j)
            if j == 0:
                o0 = o
            else:
                assert Q[s] == o0.overlap(o), (v, s)


@pytest.mark.slow
def test_full_batch_workload_every_replica(isg):
    """The 512-sample workload at the benchmark's launch configuration (the
    pass engine with two words per lane, which the autotuner picks for MT19937;
    one graph-replayed persistent launch of 64 sweeps): the tracked energy and
    the hash of all 1024 replicas and the overlap of all 512 samples against the
    oracle.  The oracles run 16 at a time on host threads (the ctypes calls
    release the interpreter lock), one thread each."""
    import concurrent.futures as cf
    import os
    from paper_1411_0127_gb300 import workloads
    samples = workloads.batch_samples()
    b = isg.Batch([x.L for x in samples], [x.seed_J for x in samples], [v for x in samples for v in x.seed_spin],
                  [1.0 / x.T for x in samples], "mt19937")
    b.set_config(4, 4, 0, 2)
    b.run(64, group_sweeps=64)
    E, Q = b.measure()
    Et, H = b.tracked()
    assert np.array_equal(E, Et)
    b.close()

    def one(s):
        x = samples[s]
        o = [OracleSim(x.L, x.seed_J, x.seed_spin[j], 1.0 / x.T, oracle.RNG_MT19937) for j in range(2)]
        for oj in o:
            oj.sweep(64, threads=1)
        r = (o[0].tracked_energy(), o[1].tracked_energy(), o[0].hash(), o[1].hash(), o[0].overlap(o[1]))
        for oj in o:
            oj.close()
        return r

    order = sorted(range(len(samples)), key=lambda s: -samples[s].L)   # largest first
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        res = dict(zip(order, ex.map(one, order)))
    for s in range(len(samples)):
        e0, e1, h0, h1, q = res[s]
        assert E[2 * s] == e0 and E[2 * s + 1] == e1, (s, samples[s].L)
        assert int(H[2 * s]) == h0 and int(H[2 * s + 1]) == h1, (s, samples[s].L)
        assert Q[s] == q, (s, samples[s].L)


def test_batch_rejects_bad_arguments(isg):
    with pytest.raises(isg.IsgError):
        isg.Batch([16, 15], [1, 2], [1, 2, 3, 4], [1.0, 1.0])
    with pytest.raises(isg.IsgError):
        isg.Batch([16], [1], [1, 2], [0.0])


@pytest.mark.parametrize("kind", ["mt19937", "minstd", "parisi_rapuano"])
def test_every_execution_configuration_gives_identical_states(isg, kind):
    """Layout and tuning invariance: each candidate the autotuner may pick (CTA
    shape, streams per bundle, generator-state placement, words per lane) sweeps the same mixed
    batch to bit-identical states (energies and hashes of every replica), also
    when the configuration changes between groups of sweeps."""
    from paper_1411_0127_gb300 import autotune
    L, J, S, B = mixed()
    ref = isg.Batch(L, J, S, B, kind)
    ref.run(6, 3)
    E0, H0 = ref.tracked()
    ref.close()
    cands = autotune.candidates()
    for cand in cands:
        b = isg.Batch(L, J, S, B, kind)
        b.set_config(*cand)
        assert b.get_config() == tuple(cand)
        b.run(6, 3)
        E, H = b.tracked()
        assert np.array_equal(E, E0) and np.array_equal(H, H0), cand
        b.close()
    # switching configurations mid-run
    b = isg.Batch(L, J, S, B, kind)
    for i, cand in enumerate(cands[:3]):
        b.set_config(*cand)
        b.run(2, 2)
    E, H = b.tracked()
    assert np.array_equal(E, E0) and np.array_equal(H, H0)
    Em, _ = b.measure()
    assert np.array_equal(Em, E0)
    b.close()


def test_autotuner_picks_a_candidate_and_caches_it(isg, tmp_path):
    from paper_1411_0127_gb300 import autotune
    L, J, S, B = mixed()
    b = isg.Batch(L, J, S, B, "mt19937")
    b.run(2, 2)
    E0, H0 = b.tracked()
    cache = str(tmp_path / "tune.json")
    res = b.autotune(sweeps=2, cache=cache)
    assert not res["cached"]
    assert tuple(res["config"]) in autotune.candidates()
    assert len(res["table"]) == len(autotune.candidates())
    assert b.get_config() == tuple(res["config"])
    E1, H1 = b.tracked()                               # the tuner ran on a twin
    assert np.array_equal(E1, E0) and np.array_equal(H1, H0)
    again = b.autotune(sweeps=2, cache=cache)
    assert again["cached"] and tuple(again["config"]) == tuple(res["config"])
    b.close()


def test_batch_config_rejects_bad_values(isg):
    L, J, S, B = mixed()
    b = isg.Batch(L[:2], J[:2], S[:4], B[:2], "minstd")
    for bad in [(6, 0, 1, 1), (-1, 0, 1, 1), (2, 17, 1, 1), (0, 33, 1, 1), (0, 8, 2, 1), (0, 8, 1, 3), (0, 8, 1, 0),
                (4, 5, 0, 1), (5, 5, 0, 1)]:
        with pytest.raises(isg.IsgError):
            b.set_config(*bad)
    assert b.get_config() == (0, 32, 1, 1)
    b.close()


def test_dependency_wait_gives_up_with_a_status(isg):
    """Failure detection without a GPU fault: the last task is made to wait for
    a flag that nothing sets.  Its bounded wait runs out, the launch ends, the
    next read reports ISG_ERR_TIMEOUT once, and the context stays usable."""
    L, J, S, B = mixed()
    b = isg.Batch(L, J, S, B, "minstd")
    assert b.info()["bundles"] >= 2
    assert isg.lib().isg_batch_test_stall(b._h) == isg.ISG_OK
    b.run(1, group_sweeps=1)
    with pytest.raises(isg.IsgError) as ex:
        b.tracked()
    assert ex.value.code == isg.ISG_ERR_TIMEOUT
    b.tracked()                                   # reported once
    b.set_config(0, 32, 1, 1)                     # a fresh plan
    b.run(2, group_sweeps=2)
    Em, _ = b.measure()
    Et, _ = b.tracked()
    assert np.array_equal(Em, Et)                 # every replica's bookkeeping intact
    b.close()


def test_pass_engine_wait_gives_up_with_a_status(isg):
    """The group pass engine's bounded wait: the pass-1 items of one lattice are made
    to wait for one completed item too many.  The wait runs out, the next read
    reports ISG_ERR_TIMEOUT once, and the context stays usable; a fresh plan
    sweeps on with every replica's bookkeeping intact."""
    L, J, S, B = mixed()
    b = isg.Batch(L, J, S, B, "minstd")
    b.set_config(4, 4, 0, 1)
    assert isg.lib().isg_batch_test_stall(b._h) == isg.ISG_ERR_STATE   # no waits in the per-pass launches
    b.set_config(5, 4, 0, 1)
    assert isg.lib().isg_batch_test_stall(b._h) == isg.ISG_OK
    b.run(1, group_sweeps=1)
    with pytest.raises(isg.IsgError) as ex:
        b.tracked()
    assert ex.value.code == isg.ISG_ERR_TIMEOUT
    b.tracked()                                   # reported once
    b.set_config(5, 4, 0, 1)                      # a fresh plan
    b.run(2, group_sweeps=2)
    Em, _ = b.measure()
    Et, _ = b.tracked()
    assert np.array_equal(Em, Et)
    b.close()


def test_member_packed_spin_io(isg):
    """Batch members keep 64-bit words whatever L; where L / 2 is an odd
    multiple of 32 (L = 64, 192) the last word of a row holds 32 valid sites.
    Packed-bit spin I/O on such members against the int8 path: read after
    sweeps, a round trip of a random configuration, tail bits left zero (the
    energy bookkeeping and the trajectory afterwards stay exact)."""
    L = [64, 192, 128]
    b = isg.Batch(L, [11, 12, 13], [21, 22, 23, 24, 25, 26], [1 / 0.9] * 3, "mt19937")
    b.run(3, group_sweeps=3)
    for r in range(2 * len(L)):
        m = b.member(r)
        n = L[r // 2]
        ref = m.read_spins()
        np.testing.assert_array_equal(m.read_spins_packed(), np.packbits(ref == 1, bitorder="little"))
        rng = np.random.default_rng(r)
        s = np.where(rng.random(n ** 3) < 0.5, 1, -1).astype(np.int8)
        m.write_spins_packed(np.packbits(s == 1, bitorder="little"))
        np.testing.assert_array_equal(m.read_spins(), s)
        assert m.tracked_energy() == m.energy()
        m.write_spins(-s)                                   # the int8 path on the same layout
        np.testing.assert_array_equal(m.read_spins_packed(), np.packbits(-s == 1, bitorder="little"))
        assert m.tracked_energy() == m.energy()
    b.run(2, group_sweeps=2)
    E, _ = b.measure()
    Et, _ = b.tracked()
    assert np.array_equal(E, Et)
    b.close()
