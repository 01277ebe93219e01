"""Asynchronous multispin coding (Sec. 4) through the C-ABI against the oracle.

Every attempt consumes one draw whatever the outcome, so system b of an ensemble
that shares one draw per site follows exactly the trajectory of a lone lattice
with the same couplings and spins and streams seeded from the ensemble's
seed_rng.  The oracle runs that lone lattice (OracleSim(..., seed_rng=R)); spins
and energies must agree bit for bit, every system, after every checked sweep.

Sizes: L = 4 (two sites per row and colour), L = 10 and 50 (ragged tails of the
32-site blocks), L = 50 and 64 (several streams), L = 256 (512 streams of 128
rows; rows of 128 sites: the staged kernel form), L = 432 (2456 streams: the
register form with four blocks of sites in flight per lane), L = 512 and 768
(staged, two and three chunks per row); beta = inf (only u >= 3 flips)."""
import math

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


def seeds(base):
    rng = np.random.default_rng(base)
    J = [int(v) for v in rng.integers(0, 2**63, 32, dtype=np.int64)]
    S = [int(v) for v in rng.integers(0, 2**63, 32, dtype=np.int64)]
    return J, S


def oracles(L, J, S, R, beta, kind):
    return [OracleSim(L, J[b], S[b], beta, kind, seed_rng=R) for b in range(32)]


@pytest.mark.parametrize("L,kind,beta,sweeps,every", [
    (4, "minstd", 1 / 1.1, 6, 1),
    (10, "mt19937", 1 / 0.7, 7, 1),
    (12, "mt19937", math.inf, 5, 1),
    (50, "minstd", 1 / 0.9, 4, 2),
    (64, "mt19937", 1 / 0.9, 3, 3),
    (10, "parisi_rapuano", 1 / 0.8, 6, 2),
    (50, "parisi_rapuano", 1 / 1.1, 4, 4),
    (256, "minstd", 1 / 0.9, 2, 1),
    (256, "parisi_rapuano", 1 / 0.7, 2, 2),
])
def test_every_system_matches_its_lone_lattice(isg, L, kind, beta, sweeps, every):
    J, S = seeds(L)
    R = 0x5EED0000 + L
    m = isg.Amsc(L, J, S, R, beta, kind)
    orc = oracles(L, J, S, R, beta, isg.RNG_KINDS[kind])
    E_prev = None
    for s in range(0, sweeps + 1, every):
        if s:
            m.sweep(every)
            for o in orc:
                o.sweep(every, threads=4)
        E = m.energies()
        for b in range(32):
            np.testing.assert_array_equal(m.spins(b), orc[b].spins(), err_msg="system %d, sweep %d" % (b, s))
            assert E[b] == orc[b].energy(), (b, s)
        if beta == math.inf and E_prev is not None:
            assert (E <= E_prev).all()
        E_prev = E
    # the 32 systems are different systems
    assert len({m.spins(b).tobytes() for b in range(32)}) == 32


def test_large_lattice_against_single_lattice_handles(isg):
    """L = 256, MT19937, 2 sweeps: systems 0, 13 and 31 against lone GPU handles
    seeded the same way (the handles are bit-exact with the oracle elsewhere);
    all 32 energies against the handles' energies."""
    L, kind, beta = 256, "mt19937", 1 / 0.7
    J, S = seeds(7)
    R = 99
    m = isg.Amsc(L, J, S, R, beta, kind)
    m.sweep(2)
    E = m.energies()
    for b in range(32):
        h = isg.Sim(L, J[b], S[b], beta, kind, seed_rng=R)
        h.sweep(2)
        assert E[b] == h.energy(), b
        if b in (0, 13, 31):
            np.testing.assert_array_equal(m.spins(b), h.read_spins())
        h.close()


@pytest.mark.parametrize("L,kind,sweeps,form", [
    (432, "mt19937", 3, 4), (432, "parisi_rapuano", 2, 4),
    (512, "minstd", 2, 0), (512, "parisi_rapuano", 2, 0), (768, "mt19937", 2, 0),
])
def test_large_ensembles_against_lone_lattices_and_oracle(isg, L, kind, sweeps, form):
    """The kernel forms of large ensembles: the register form with four blocks
    of 32 sites in flight per lane (at least 16 streams per SM and rows that are
    not a multiple of 128 sites: L = 432, 2456 streams, a 32-site tail block in
    every stream) and the staged form (rows of a multiple of 128 sites, fetched
    by bulk copies: L = 512 with two chunks per row, L = 768 with three, so both
    row wraps and interior chunks).  All 32 energies against lone GPU handles
    seeded the same way, the spins of systems 0, 13 and 31 against those
    handles, and system 5 directly against the oracle."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    beta = 1 / 0.9
    J, S = seeds(L + 1)
    R = 0xA5C0 + L
    m = isg.Amsc(L, J, S, R, beta, kind)
    info = m.info()
    assert info["form"] == form, info
    if form == 4:
        assert info["streams"] >= 16 * sms, info
    m.sweep(sweeps)
    E = m.energies()
    for b in range(32):
        h = isg.Sim(L, J[b], S[b], beta, kind, seed_rng=R)
        h.sweep(sweeps)
        assert E[b] == h.energy(), (b, kind)
        if b in (0, 13, 31):
            np.testing.assert_array_equal(m.spins(b), h.read_spins(), err_msg="system %d" % b)
        h.close()
    o = OracleSim(L, J[5], S[5], beta, isg.RNG_KINDS[kind], seed_rng=R)
    o.sweep(sweeps, threads=16)
    np.testing.assert_array_equal(m.spins(5), o.spins())
    assert E[5] == o.energy() == o.tracked_energy()
    o.close()
    m.close()


def test_shared_draws_make_identical_systems_move_together(isg):
    """32 copies of one system (same couplings and spins) stay identical: the
    draw is shared, so the broadcast cond masks flip every copy alike."""
    J, S = [5] * 32, [6] * 32
    m = isg.Amsc(16, J, S, 17, 1 / 1.1, "mt19937")
    m.sweep(5)
    ref = m.spins(0)
    for b in range(1, 32):
        np.testing.assert_array_equal(m.spins(b), ref)
    assert len(set(m.energies().tolist())) == 1


def test_read_spins_rejects_bad_sample(isg):
    J, S = seeds(1)
    m = isg.Amsc(8, J, S, 1, 1.0, "minstd")
    with pytest.raises(isg.IsgError):
        m.spins(32)
    with pytest.raises(isg.IsgError):
        m.sweep(-1)
