"""helm_precond_apply_noalloc: the allocation-free V-cycle entry point.

It exists for callers that cannot let a library call cudaMalloc (device memory
reserved up front by a pooling allocator, or loops that cannot afford the device
synchronisation of cudaMalloc/cudaFree).  Its working memory is a fixed array inside
the library.  These tests call it through the C ABI twice in a row and compare each
result with the allocating entry point (helm_precond_apply on a handle) within the
V-cycle parity tolerances of the other GPU tests (c64 5e-5, c128 1e-11 relative); they
also check that free device memory does not move across calls, and that a grid too
large for the fixed array is rejected.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1012_5379_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_5379_gb300 import build, helm as H
    build.build()
    H.load()
    return H


def rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,n,prec,tol", [(2, 63, "c64", 5e-5), (2, 127, "c64", 5e-5),
                                            (3, 15, "c128", 1e-11), (2, 31, "c128", 1e-11)])
def test_noalloc_matches_allocating_entry_point(helm, dim, n, prec, tol):
    k, tb = 0.15 * (n + 1), 0.3
    dt = torch.complex64 if prec == "c64" else torch.complex128
    h = helm.Handle(dim, n, tb, k=k, precision=prec, maxit=1)
    outs = []
    for seed in (11, 12):  # two calls in a row, different inputs
        r = torch.from_numpy(I.random_source(dim, n, seed)).cuda().to(dt)
        want = torch.empty_like(r)
        h.precond_apply(r, want)
        got = torch.full_like(r, float("nan"))
        helm.precond_apply_noalloc(dim, n, tb, k, r, got, precision=prec)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(got)).all()
        assert rel(got, want) < tol
        outs.append(got)
    assert not torch.equal(outs[0], outs[1])


def test_noalloc_allocates_no_device_memory(helm):
    dim, n, k, tb = 2, 63, 10.0, 0.3
    r = torch.from_numpy(I.random_source(dim, n, 3)).cuda().to(torch.complex64)
    z = torch.empty_like(r)
    helm.precond_apply_noalloc(dim, n, tb, k, r, z)   # first call: resolves the array address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        helm.precond_apply_noalloc(dim, n, tb, k, r, z)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_grids_beyond_its_array(helm):
    r = torch.zeros((255, 255), dtype=torch.complex64, device="cuda")
    z = torch.empty_like(r)
    with pytest.raises(helm.HelmError) as e:
        helm.precond_apply_noalloc(2, 255, 0.3, 10.0, r, z)
    assert e.value.code == helm.HELM_EINVAL and "bytes of scratch" in str(e.value)
