"""CPU checks of the boundary: the library builds for sm_103a, loads, and exports every
entry point that include/rchfsi.h declares (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rchfsi.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int64_t|int)\s+(rcf_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_30128_gb300.build import build
    return build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for need in ("rcf_create", "rcf_mesh_create", "rcf_potential_set", "rcf_projectors_set",
                 "rcf_filter", "rcf_residual", "rcf_rayleigh_ritz", "rcf_adjoint_filter",
                 "rcf_lanczos_bounds", "rcf_apply", "rcf_status_string", "rcf_last_error"):
        assert need in syms


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing


def test_binding_lists_every_symbol(libpath):
    from paper_2605_30128_gb300 import rchfsi
    assert sorted(rchfsi.EXPORTS) == declared_symbols()
    L = rchfsi.lib()
    assert L.rcf_status_string(0) == b"ok"
    assert L.rcf_status_string(4).startswith(b"Gram")


def test_null_arguments_are_rejected_without_a_gpu(libpath):
    from paper_2605_30128_gb300 import rchfsi as R
    L = R.lib()
    assert L.rcf_create(None, 0, None) == R.RCF_EINVAL
    assert L.rcf_mesh_info(None, None, None, None) == R.RCF_EINVAL
    assert L.rcf_filter(None, None, None, 0, 0, None, 1, None, 0, 0, 0, None, 0) == R.RCF_EINVAL


def test_bfp_stream_size_without_a_gpu(libpath):
    from oracle.bfp import bfp_stream_bytes
    from paper_2605_30128_gb300 import rchfsi as R
    for nbits in R.RCF_BFP_RATES:
        for n in (0, 1, 3, 4, 5, 1023, 1 << 33):
            assert R.rcf_bfp_stream_bytes(n, nbits) == bfp_stream_bytes(n, nbits)
    L = R.lib()
    assert L.rcf_bfp_stream_bytes(4, 8) == -1 and L.rcf_bfp_stream_bytes(-1, 16) == -1
    assert L.rcf_bfp_encode(None, None, 4, 16, None) == R.RCF_EINVAL
    assert L.rcf_bfp_decode(None, None, 4, 16, None) == R.RCF_EINVAL
