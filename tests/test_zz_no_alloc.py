"""The allocation-free run entry point gives the same lattice as the handle path.

ac_run_blocked_static serves callers that cannot let the library allocate
device memory: an application whose own memory pool reserved the device up
front, a host that gives the library a fixed device budget, or a loop that must
not call cudaMalloc / cudaFree because they can synchronise the device.  It
keeps its working buffers in a fixed file-scope device array.  This test feeds
it a lattice held in torch-owned device buffers and compares, on two calls in a
row, with a handle run through ac_run_until_ticks: bit-exact, the tolerance of
every parity test here.  It also checks that a lattice too large for the fixed array is refused.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

T32 = 1 << 32


def _packed_state(sim):
    """(key, cnt) device tensors of a handle's state: key = tick << 1 | (spin > 0)."""
    N = sim.rows * sim.cols
    s = torch.empty(N, dtype=torch.int8, device="cuda")
    t = torch.empty(N, dtype=torch.int64, device="cuda")
    n = torch.empty(N, dtype=torch.int32, device="cuda")
    ac.ac_read_state_device(sim.handle, s.data_ptr(), t.data_ptr(), n.data_ptr())
    key = t * 2 + (s > 0).to(torch.int64)
    return key, n


@pytest.mark.parametrize("rows,cols,beta,h,seed", [(300, 260, 0.44, 0.0, 5), (64, 64, 0.6, 0.1, 1),
                                                   (2, 130, 0.3, -0.2, 9)])
def test_static_entry_matches_handle_on_two_calls(rows, cols, beta, h, seed):
    with ac.Sim(rows, cols, beta, 1.0, h, seed, kernel=ac.AC_KERNEL_BLOCKED, Lb=64) as ref:
        key, cnt = _packed_state(ref)            # caller-owned copies of the initial state
        for T in (2, 5):
            ref.run_until_ticks(T * T32)
            ac.ac_run_blocked_static(rows, cols, beta, 1.0, h, seed, key.data_ptr(), cnt.data_ptr(), T * T32)
            torch.cuda.synchronize()
            want_key, want_cnt = _packed_state(ref)
            assert torch.equal(key, want_key), f"keys differ after T={T}"
            assert torch.equal(cnt, want_cnt), f"counts differ after T={T}"


def test_static_entry_refuses_lattices_beyond_its_scratch():
    key = torch.zeros(4, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(ac.ACError) as ei:
        ac.ac_run_blocked_static(4096, 4096, 0.44, 1.0, 0.0, 1, key.data_ptr(), cnt.data_ptr(), T32)
    assert ei.value.status == ac.ac.AC_ERR_ARG
    assert "maximum" in str(ei.value)
