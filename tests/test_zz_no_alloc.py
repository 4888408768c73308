"""p4d_jvp_noalloc: the coupled JVP for callers that cannot allocate device
memory when they call it (inside CUDA stream capture, or with all device
memory owned by a framework's pool).  Its one scratch array is a fixed
device array of the library; the result must equal p4d_jvp's.

Collected last on purpose (file name) so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from p4d_inputs import make_case, make_box_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07225_gb300 import build, _native
    build.build()
    return _native.load()


def _field_rel(s, a, b):
    nn = s.nn
    out = []
    for sl in (slice(0, nn), slice(nn, 2 * nn), slice(2 * nn, 3 * nn), slice(3 * nn, s.ndof)):
        nb = np.linalg.norm(b[sl])
        out.append(np.linalg.norm(a[sl] - b[sl]) / (nb if nb > 0 else 1.0))
    return max(out)


@pytest.mark.parametrize("name", ["cube8", "hetero"])
@pytest.mark.parametrize("transpose", [0, 1])
def test_noalloc_jvp_matches_jvp_twice(lib, name, transpose):
    from paper_2602_07225_gb300 import P4DSolver
    case = make_case("cube8") if name == "cube8" else make_box_case(
        8, 8, (6, 4, 6), 60e-6, (60e-6, 25e-6, 60e-6), 6, 1234, hetero=True, rs_cv=0.3)
    s = P4DSolver(case, precision=1)
    st = s.state_tensors(case["state"])
    s.jacobian_update(st)
    rng = np.random.default_rng(21)
    for call in range(2):
        x = torch.tensor(rng.standard_normal(s.ndof), device="cuda")
        y_ref = s.jvp(x, transpose=bool(transpose))
        y = torch.full_like(x, float("nan"))
        st_ = lib.p4d_jvp_noalloc(s.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), transpose)
        torch.cuda.synchronize()
        assert st_ == 0, st_
        assert _field_rel(s, y.cpu().numpy(), y_ref.cpu().numpy()) < 1e-11, call


@pytest.mark.parametrize("transpose", [0, 1])
def test_noalloc_jvp_under_stream_capture(lib, transpose):
    """The use the entry point exists for: a call captured into a CUDA graph
    on the handle's stream (after one eager call), the graph replayed on new
    contents of the captured input buffer."""
    from paper_2602_07225_gb300 import P4DSolver
    case = make_case("cube8")
    cs = torch.cuda.Stream()
    s = P4DSolver(case, precision=1, stream=cs)
    with torch.cuda.stream(cs):
        st = s.state_tensors(case["state"])
        s.jacobian_update(st)
        x = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        assert lib.p4d_jvp_noalloc(s.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), transpose) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        rc = lib.p4d_jvp_noalloc(s.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), transpose)
    assert rc == 0, rc
    rng = np.random.default_rng(22)
    for _ in range(2):
        x.copy_(torch.tensor(rng.standard_normal(s.ndof), device="cuda"))
        y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        y_ref = s.jvp(x, transpose=bool(transpose))
        torch.cuda.synchronize()
        assert _field_rel(s, y.cpu().numpy(), y_ref.cpu().numpy()) < 1e-11


def test_noalloc_rejects_too_many_electrode_nodes(lib):
    """cube128 has 1,364,562 electrode nodes > P4D_NOALLOC_MAX_NELEC = 2^20."""
    from paper_2602_07225_gb300 import P4DSolver
    case = make_case("cube128")
    s = P4DSolver(case, precision=1)
    assert s.NE > (1 << 20)
    st = s.state_tensors(case["state"])
    s.jacobian_update(st)
    x = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert lib.p4d_jvp_noalloc(s.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), 0) == 1
    s.close()
