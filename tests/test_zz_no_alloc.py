"""isg_energy_static_scratch: the energy for callers that must not allocate.

Some callers cannot let the library call cudaMalloc when they ask for the
energy: real-time loops that cannot take the device-wide synchronisation an
allocation may cause, and processes or embedding runtimes that work inside a
device-memory budget fixed up front.  This entry point keeps its scratch in a
fixed array compiled into the library; here it is called through the C-ABI and
must give exactly the value isg_energy gives and the oracle's energy of the
same trajectory (integer energies: tolerance zero), on two calls in a row and
again after more sweeps.  The file is named so that pytest collects it after
every other test file.
"""
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


def _static_energy(isg, sim, out, stream):
    rc = isg.lib().isg_energy_static_scratch(sim.handle, out.data_ptr(), stream.cuda_stream)
    assert rc == isg.ISG_OK, isg.lib().isg_last_error()


@pytest.mark.parametrize("L,kind", [(64, "mt19937"), (130, "minstd"), (256, "mt19937")])
def test_static_scratch_energy_equals_isg_energy(isg, L, kind):
    import torch
    stream = torch.cuda.current_stream()
    beta = 1 / 0.9
    sim = isg.Sim(L, 3, 4, beta, kind)
    orc = OracleSim(L, 3, 4, beta, isg.RNG_KINDS[kind])
    out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    sim.sweep(3, stream)
    orc.sweep(3, threads=8)
    _static_energy(isg, sim, out[0], stream)          # two calls in a row
    _static_energy(isg, sim, out[1], stream)
    torch.cuda.synchronize()
    E = sim.energy(stream)
    assert int(out[0].item()) == E == orc.energy()
    assert int(out[1].item()) == E
    sim.sweep(5, stream)                               # the shared array is reused
    orc.sweep(5, threads=8)
    _static_energy(isg, sim, out[2], stream)
    _static_energy(isg, sim, out[3], stream)
    torch.cuda.synchronize()
    E2 = sim.energy(stream)
    assert int(out[2].item()) == E2 == int(out[3].item())
    assert E2 == sim.tracked_energy() == orc.energy()
    sim.close()
    orc.close()


def test_static_scratch_rejects_lattices_beyond_its_array(isg):
    import torch
    sim = isg.Sim(1450, 1, 2, 1.0, "minstd")           # needs 8214 partial sums > 8192
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = isg.lib().isg_energy_static_scratch(sim.handle, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == isg.ISG_ERR_ARG
    assert b"1448" in isg.lib().isg_last_error()
    sim.close()
