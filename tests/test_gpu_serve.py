"""Request server (continuous batching) on the GPU: every job served in a mix
of concurrent jobs must give exactly the result it gives alone (energy and
Zobrist hash equal; tolerance zero), whatever the budget, quantum or number of
jobs on the device at once."""
import numpy as np
import pytest

from oracle import OracleSim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_0127_gb300 import build
    build.build()
    import paper_1411_0127_gb300 as m
    return m


def trace(n=28, seed=3):
    rng = np.random.default_rng(seed)
    sizes = [32, 48, 64, 96, 128, 224, 256]
    jobs = []
    t = 0.0
    for j in range(n):
        t += rng.exponential(0.01)
        jobs.append(dict(L=int(rng.choice(sizes)), seed_J=700 + j, seed_spin=900 + j,
                         beta=1.0 / float(rng.uniform(0.5, 1.5)), kind=("minstd", "mt19937", "parisi_rapuano")[j % 3],
                         sweeps=int(rng.integers(5, 120)), arrival=t))
    return jobs


def alone(isg, job):
    s = isg.Sim(job["L"], job["seed_J"], job["seed_spin"], job["beta"], job["kind"])
    s.sweep(job["sweeps"])
    out = (s.energy(), s.hash(), s.tracked_energy())
    s.close()
    return out


@pytest.fixture(scope="module")
def reference(isg):
    return {j: alone(isg, job) for j, job in enumerate(trace())}


@pytest.mark.parametrize("budget,quantum,max_active", [(150 * 10**9, 16, 4096), (60 * 10**6, 7, 4096),
                                                       (150 * 10**9, 64, 1)])
def test_served_jobs_equal_alone(isg, reference, budget, quantum, max_active):
    jobs = trace()
    srv = isg.Server(budget, quantum, max_active)
    ids = [srv.submit(j["L"], j["seed_J"], j["seed_spin"], j["beta"], j["kind"], j["sweeps"], j["arrival"])
           for j in jobs]
    srv.run(time_limit_s=300)
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    if max_active == 1:
        assert st["peak_active"] == 1
    for j, jid in enumerate(ids):
        r = srv.job(jid)
        assert r["status"] == 2, (j, r)
        E, H, Et = reference[j]
        assert r["E"] == E == Et, (j, jobs[j])
        assert r["H"] == H, (j, jobs[j])
        assert r["done"] >= r["admit"] >= r["arrival"] - 1e-9
    srv.close()


def test_served_jobs_match_oracle(isg):
    jobs = [dict(L=32, seed_J=5, seed_spin=6, beta=1 / 0.8, kind="mt19937", sweeps=40, arrival=0.0),
            dict(L=48, seed_J=7, seed_spin=8, beta=1 / 1.3, kind="minstd", sweeps=25, arrival=0.001),
            dict(L=36, seed_J=9, seed_spin=10, beta=1 / 1.0, kind="mt19937", sweeps=33, arrival=0.002),
            dict(L=40, seed_J=11, seed_spin=12, beta=1 / 0.9, kind="parisi_rapuano", sweeps=29, arrival=0.003)]
    srv = isg.Server(10**10, 10, 16)
    ids = [srv.submit(j["L"], j["seed_J"], j["seed_spin"], j["beta"], j["kind"], j["sweeps"], j["arrival"])
           for j in jobs]
    srv.run(60)
    for jid, j in zip(ids, jobs):
        o = OracleSim(j["L"], j["seed_J"], j["seed_spin"], j["beta"], isg.RNG_KINDS[j["kind"]])
        o.sweep(j["sweeps"])
        r = srv.job(jid)
        assert r["E"] == o.energy() and r["H"] == o.hash(), j
    srv.close()


def test_server_rejects_bad_jobs(isg):
    srv = isg.Server(10 * 10**6, 16, 8)
    with pytest.raises(isg.IsgError):
        srv.submit(512, 1, 2, 1.0, "mt19937", 10, 0.0)     # larger than the whole budget
    with pytest.raises(isg.IsgError):
        srv.submit(33, 1, 2, 1.0, "mt19937", 10, 0.0)
    with pytest.raises(isg.IsgError):
        srv.submit(32, 1, 2, 0.0, "mt19937", 10, 0.0)
    srv.run(5)                                              # nothing queued: returns at once
    srv.close()
