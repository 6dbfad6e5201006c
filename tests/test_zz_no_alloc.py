"""helm_precond_apply_noalloc: the allocation-free V-cycle entry point.

It exists for callers that cannot let a library call cudaMalloc (device memory
reserved up front by a pooling allocator, or loops that cannot afford the device
synchronisation of cudaMalloc/cudaFree).  Its working memory is a fixed array inside
the library.  These tests call it through the C ABI twice in a row and compare each
result with the allocating entry point (helm_precond_apply on a handle) and with the
FP64 oracle's V-cycle, within the V-cycle parity tolerances of the other GPU tests
(relative 2-norm and worst point, c64 5e-5, c128 1e-11; tests/parity_check.py), up to
the largest grids the array holds; they also check that free device memory does not
move across calls, that grids too large for the fixed array, a coarsest level above
32 unknowns and mismatched tensors are rejected.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_1012_5379_gb300 import inputs as I
from parity_check import assert_parity

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


@pytest.mark.parametrize("dim,n,prec", [(2, 63, "c64"), (2, 127, "c64"), (3, 15, "c128"), (2, 31, "c128"),
                                        (3, 31, "c64"), (2, 127, "c128")])
def test_noalloc_matches_allocating_entry_point_and_oracle(helm, dim, n, prec):
    k, tb = 0.15 * (n + 1), 0.3
    dt = torch.complex64 if prec == "c64" else torch.complex128
    h = helm.Handle(dim, n, tb, k=k, precision=prec, maxit=1)
    levels = O.build_hierarchy(dim, n, tb, I.THETA_GAMMA, I.ECS_FRAC, k=k)
    outs = []
    for seed in (11, 12):  # two calls in a row, different inputs
        src = I.random_source(dim, n, seed)
        r = torch.from_numpy(src).cuda().to(dt)
        want = torch.empty_like(r)
        h.precond_apply(r, want)
        got = torch.full_like(r, float("nan"))
        helm.precond_apply_noalloc(dim, n, tb, k, r, got, precision=prec)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(got)).all()
        assert_parity(got, want, ("vcycle", prec), "vs helm_precond_apply")
        assert_parity(got, O.vcycle(levels, r.cpu().numpy().astype(np.complex128)), ("vcycle", prec), "vs oracle")
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
    for dim, n, prec in ((2, 255, "c64"), (3, 31, "c128")):
        dt = torch.complex64 if prec == "c64" else torch.complex128
        r = torch.zeros((n,) * dim, dtype=dt, device="cuda")
        z = torch.empty_like(r)
        with pytest.raises(helm.HelmError) as e:
            helm.precond_apply_noalloc(dim, n, 0.3, 10.0, r, z, precision=prec)
        assert e.value.code == helm.HELM_EINVAL and "bytes of scratch" in str(e.value)


def test_noalloc_rejects_a_coarsest_level_above_32_unknowns(helm):
    r = torch.zeros((63, 63), dtype=torch.complex64, device="cuda")
    z = torch.empty_like(r)
    with pytest.raises(helm.HelmError) as e:
        helm.precond_apply_noalloc(2, 63, 0.3, 10.0, r, z, coarsest_n=7)   # 7^2 = 49 unknowns
    assert e.value.code == helm.HELM_EINVAL and "32 unknowns" in str(e.value)


def test_noalloc_rejects_mismatched_tensors_before_any_launch(helm):
    n0 = helm.launch_count()
    r = torch.zeros((31, 31), dtype=torch.complex128, device="cuda")
    for z in (torch.empty((31, 31), dtype=torch.complex64, device="cuda"),    # precision
              torch.empty((31, 30), dtype=torch.complex128, device="cuda"),   # shape
              torch.empty((31, 62), dtype=torch.complex128, device="cuda")[:, ::2]):  # strides
        with pytest.raises(ValueError):
            helm.precond_apply_noalloc(2, 31, 0.3, 5.0, r, z)
    assert helm.launch_count() == n0
