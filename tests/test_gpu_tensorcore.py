"""GPU tests of the tensor-core path: the tcgen05 layout self-test (exact integer product)."""
import numpy as np
import pytest
import torch

from paper_1702_01904_gb300 import prism as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    from paper_1702_01904_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


def test_tcgen05_single_mma_exact():
    out = torch.zeros((128, 16), dtype=torch.float32, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    P.prism_selftest_tcgen05(out, st, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert int(st[0]) == 0, "MMA did not complete"
    m = np.arange(128)[:, None]
    k = np.arange(16)[None, :]
    A = ((m + 3 * k) % 7 - 3).astype(np.float64)
    n = np.arange(16)[:, None]
    B = ((5 * n + k) % 5 - 2).astype(np.float64)
    assert np.array_equal(out.cpu().numpy(), (A @ B.T).astype(np.float32))


def test_bounded_wait_runs_out_reports_and_leaves_the_context_usable():
    # failure detection without a fault: a wait that nothing completes gives up after its clock
    # budget (about 1 ms here) and reports; with its arrival the same wait completes
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    P.prism_selftest_bounded_wait(st, 2_000_000, 0, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert int(st[0]) == 1, "the wait should have run out"
    st.zero_()
    P.prism_selftest_bounded_wait(st, 2_000_000, 1, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert int(st[0]) == 0, "the completed wait should not report"
    # the context still runs the tensor-core self-test exactly
    test_tcgen05_single_mma_exact()
