"""CPU checks of the Python binding's argument validation: tensors the kernels would
read or write out of bounds (wrong precision, shape, strides, or not on the GPU) are
refused with ValueError before the C ABI is called, and the binding's constants match
include/helm.h.  No GPU is needed: the checks run before any device work."""
import os
import re

import pytest

from paper_1012_5379_gb300 import helm as H

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_define(name):
    hdr = open(os.path.join(ROOT, "include", "helm.h")).read()
    return int(re.search(rf"#define {name} (-?\d+)", hdr).group(1))


def test_constants_match_the_header():
    for name in ("HELM_C64", "HELM_C128", "HELM_CAUTO", "HELM_AUTO_C128_POINTS", "HELM_EINVAL", "HELM_ENUMERIC",
                 "HELM_ETIMEOUT"):
        assert getattr(H, name) == header_define(name), name


def test_noalloc_refuses_mismatched_precisions():
    r = torch.zeros((31, 31), dtype=torch.complex128)
    z = torch.zeros((31, 31), dtype=torch.complex64)
    with pytest.raises(ValueError, match="complex128"):
        H.precond_apply_noalloc(2, 31, 0.3, 5.0, r, z)


def test_noalloc_refuses_wrong_shapes_strides_and_host_tensors():
    r = torch.zeros((31, 31), dtype=torch.complex64)
    with pytest.raises(ValueError, match="shape"):
        H.precond_apply_noalloc(2, 31, 0.3, 5.0, r, torch.zeros((31, 30), dtype=torch.complex64))
    with pytest.raises(ValueError, match="shape"):
        H.precond_apply_noalloc(2, 31, 0.3, 5.0, r, torch.zeros(31 * 31, dtype=torch.complex64))
    with pytest.raises(ValueError, match="contiguous"):
        H.precond_apply_noalloc(2, 31, 0.3, 5.0, r, torch.zeros((31, 62), dtype=torch.complex64)[:, ::2])
    with pytest.raises(ValueError, match="CUDA"):
        H.precond_apply_noalloc(2, 31, 0.3, 5.0, r, torch.zeros((31, 31), dtype=torch.complex64))
    with pytest.raises(ValueError, match="complex64 or complex128"):
        H.precond_apply_noalloc(2, 31, 0.3, 5.0, r.real.contiguous(), r.real.contiguous())


def test_vector_checks_of_handle_calls():
    """The checks Handle.precond_apply / apply_operator / solve run first (a handle is
    not needed to exercise them)."""
    with pytest.raises(ValueError, match="complex128"):
        H._require_vec("b", torch.zeros((15, 15), dtype=torch.complex64), (15, 15), "c128")
    with pytest.raises(ValueError, match="shape"):
        H._require_vec("r", torch.zeros((15, 14), dtype=torch.complex64), (15, 15))
    H._require_vec("r", 12345, (15, 15))   # raw pointers pass unchecked


def test_unknown_precision_is_refused():
    with pytest.raises(ValueError):
        H._precision_code("fp16")
    assert H._precision_code("auto") == header_define("HELM_CAUTO")
