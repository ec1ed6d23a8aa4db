"""rihf_eigh_noalloc: the eigensolver for callers that cannot allocate device
memory (for example an MD engine that owns a fixed pool and forbids cudaMalloc
inside its time loop).  Through the C ABI, on caller-owned device buffers, two
calls in a row must reproduce the allocating entry point rihf_eigh; orders
above the fixed workspace's limit (256) must be rejected.

Collected last on purpose (file name), so a failure here leaves every other test
already run; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sym(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.normal(size=(n, n))
    return (M + M.T) / 2 + np.diag(np.linspace(-2.0, 2.0, n))


def _noalloc(R, torch, A):
    n = A.shape[0]
    dA = torch.tensor(A, dtype=torch.float64, device="cuda")
    dW = torch.empty(n, dtype=torch.float64, device="cuda")
    dV = torch.empty((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = R.eigh_noalloc(n, dA.data_ptr(), dW.data_ptr(), dV.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, dW.cpu().numpy(), dV.cpu().numpy()


def test_noalloc_matches_allocating_eigh_twice():
    torch = pytest.importorskip("torch")
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    for n, seed in [(200, 1), (37, 2), (256, 3)]:   # later calls reuse the shared workspace; 256 is the limit
        A = _sym(n, seed)
        rc, W, V = _noalloc(R, torch, A)
        assert rc == 0
        Wr, Vr = R.eigh(A)
        scale = np.abs(Wr).max()
        assert np.abs(W - Wr).max() <= 1e-12 * scale
        # eigenvectors agree up to sign (the spectra here are non-degenerate)
        sgn = np.sign(np.sum(V * Vr, axis=0))
        assert np.abs(V * sgn - Vr).max() <= 1e-9
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
        assert np.abs(A @ V - V * W).max() <= 1e-11 * scale


def test_noalloc_rejects_orders_beyond_its_workspace():
    torch = pytest.importorskip("torch")
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    n = 300
    d = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert R.eigh_noalloc(n, d.data_ptr(), w.data_ptr(), d.data_ptr(), 0) == -1


def test_noalloc_allocates_no_device_memory():
    """After a first call (which resolves the workspace address), further calls,
    also on a non-default stream, leave the device's free memory unchanged."""
    torch = pytest.importorskip("torch")
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    n = 128
    A = _sym(n, 4)
    dA = torch.tensor(A, dtype=torch.float64, device="cuda")
    dW = torch.empty(n, dtype=torch.float64, device="cuda")
    dV = torch.empty((n, n), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    assert R.eigh_noalloc(n, dA.data_ptr(), dW.data_ptr(), dV.data_ptr(), side.cuda_stream) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for stream in (side.cuda_stream, torch.cuda.current_stream().cuda_stream):
        assert R.eigh_noalloc(n, dA.data_ptr(), dW.data_ptr(), dV.data_ptr(), stream) == 0
        torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    Wr, _ = R.eigh(A)
    assert np.abs(dW.cpu().numpy() - Wr).max() <= 1e-12 * np.abs(Wr).max()
