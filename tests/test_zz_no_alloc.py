"""grf_rk4_step_noalloc: the RK4 step for callers that cannot allocate device memory (code
inside a captured CUDA graph region, host frameworks that own every allocation, embedded
callers that forbid allocation after start-up). It keeps its scratch in a fixed device array
inside the library instead of a caller-provided workspace; its results must equal those of
grf_rk4_step with a workspace, call after call (the shared array keeps the previous call's
contents, which must not leak into the next result).

This file is collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import grf_inputs as gi
from parity import describe, field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_06225_gb300 import build
    build.build()
    import paper_2309_06225_gb300 as grf
    grf.lib()
    return grf


@pytest.mark.parametrize("bc", [gi.BC_PERIODIC, gi.BC_FROZEN])
def test_noalloc_matches_workspace_path_on_two_calls_in_a_row(g, bc):
    box = gi.Box(20, 14, 17, 0.3, -2.8, -2.0, -2.4, bc=bc)
    params = g.params_like(gi.Params(lam=0.2, g2=0.1, beta_kind=1))
    s0 = gi.random_perturbed_state(box, 77, base=gi.single_puncture(box, amp=0.05), eps=2e-2)
    b = g.box_like(box)
    dt = 0.25 * box.dx
    ref = g.to_device(s0, b)
    got = g.to_device(s0, b)
    for call in range(2):
        g.grf_rk4_step(b, params, ref, dt, 2)
        g.grf_rk4_step_noalloc(b, params, got, dt, 2)
        r, o = g.to_host(ref, b), g.to_host(got, b)
        errs = field_errors(o, r, box)
        assert np.max(errs) <= 1e-11, (call, describe(errs))
        assert np.array_equal(o, r), call  # same kernels, same order: bit-identical
    assert g.grf_check_status() == 0


def test_noalloc_rejects_boxes_beyond_the_fixed_scratch(g):
    big = g.make_box(40, 40, 40, 0.2)  # 3 states of 46^2 x 48 x 27 doubles > 48 MiB
    assert g.grf_workspace_bytes(big, g.GRF_OP_RK4) > g.GRF_NOALLOC_SCRATCH_BYTES
    t = g.alloc_state(big)
    with pytest.raises(g.GrfError) as e:
        g.grf_rk4_step_noalloc(big, g.params_like(gi.Params()), t, 0.05, 1)
    assert e.value.code == g.GRF_ETOOLARGE
    assert "fixed scratch" in g.grf_error_string(g.GRF_ETOOLARGE)
