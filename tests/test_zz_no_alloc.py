"""okr_power_flow_static: the load flow for callers that cannot allocate device
memory, checked through the C ABI against okr_power_flow (the context entry
point) on two calls in a row with different feeders, so that contents left in
the shared static scratch by the first call cannot leak into the second.

Collected last on purpose: it must pass alone in a fresh process and after the
other tests (the static scratch's device address is looked up on the first call
in the process, whichever test makes it).
"""
from __future__ import annotations

import numpy as np
import pytest

import feedergen as fg

pytestmark = pytest.mark.gpu

V_TOL = 1e-9          # p.u., voltages (same bound as the other GPU parity tests)
I_TOL = 1e-9          # injections


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    c = K.Context(0)
    yield c
    c.close()


def _static_run(f):
    """Feeder to the device (the test allocates; the entry point does not), then
    okr_power_flow_static on torch's current stream."""
    import torch
    import paper_2510_19608_gb300 as K
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.parent, f.phases, f.z_line, f.s_load)]
    L, n = f.n_scen, f.n_bus
    vh = torch.full((L, n, 3, 2), float("nan"), dtype=torch.float64, device="cuda")
    ih = torch.full((L, n, 3, 2), float("nan"), dtype=torch.float64, device="cuda")
    df = K.device_feeder(n, L, *[t.data_ptr() for t in dev], f.v_slack)
    torch.cuda.synchronize()
    sw = K.power_flow_static(df, vh.data_ptr(), ih.data_ptr(), torch.cuda.current_stream().cuda_stream)
    v = vh.cpu().numpy()
    i = ih.cpu().numpy()
    return v[..., 0] + 1j * v[..., 1], i[..., 0] + 1j * i[..., 1], sw


def test_static_load_flow_matches_context_entry_two_calls(ctx):
    big, _ = fg.preset("feeder1000")
    small, _ = fg.preset("feeder40")
    for f in (big, small):                      # two calls in a row, the second smaller
        v_ref, i_ref, sw_ref = ctx.power_flow(f)
        v, i, sw = _static_run(f)
        assert np.isfinite(v).all() and np.isfinite(i).all()
        assert np.abs(v - v_ref).max() <= V_TOL
        assert np.abs(i - i_ref).max() <= I_TOL
        assert sw == sw_ref


def test_static_load_flow_at_the_size_limits(ctx):
    """The largest feeder the static scratch holds (OKR_STATIC_MAX_BUS buses,
    4 scenarios: the carve fills the array exactly) and a 3,000-bus feeder
    (above the 2,048 buses whose load-flow slices fit shared memory, so the
    global-memory path of the sweep runs), each against okr_power_flow."""
    from paper_2510_19608_gb300 import _binding as B
    for n, L, seed in ((B.STATIC_MAX_BUS, 4, 4096), (3000, 2, 3000)):
        f = fg.make_feeder(n, seed, phase_mode=(0.45, 0.15, 0.4), load=("lognormal", 15.0, 1.0), n_scen=L)
        v_ref, i_ref, sw_ref = ctx.power_flow(f)
        v, i, sw = _static_run(f)
        assert np.isfinite(v).all() and np.isfinite(i).all()
        assert np.abs(v - v_ref).max() <= V_TOL
        assert np.abs(i - i_ref).max() <= I_TOL
        assert sw == sw_ref


def test_static_load_flow_reports_a_singular_line_as_the_context_entry_does(ctx):
    """A line whose impedance block is singular: both entry points return
    OKR_ESINGULAR (the static one stops after the line inverses, before its
    load flow could overwrite the flag), and the next call works."""
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import _binding as B
    f, _ = fg.preset("feeder40")
    bad = fg.Feeder(parent=f.parent.copy(), phases=f.phases.copy(), z_line=f.z_line.copy(),
                    s_load=f.s_load.copy(), v_slack=f.v_slack, meta={})
    bad.z_line[3] = 0.0
    with pytest.raises(K.OkrError) as e:
        ctx.power_flow(bad)
    assert e.value.status == B.ESINGULAR
    with pytest.raises(K.OkrError) as e:
        _static_run(bad)
    assert e.value.status == B.ESINGULAR
    v_ref, _, _ = ctx.power_flow(f)
    v, _, _ = _static_run(f)
    assert np.abs(v - v_ref).max() <= V_TOL


def test_static_load_flow_rejects_oversized_feeder():
    import torch
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import _binding as B
    n = 4097                                    # OKR_STATIC_MAX_BUS + 1: refused before any device work
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    ibuf = torch.zeros(8, dtype=torch.int32, device="cuda")
    df = K.device_feeder(n, 2, ibuf.data_ptr(), ibuf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                         np.zeros((3, 2)))
    with pytest.raises(K.OkrError) as e:
        K.power_flow_static(df, buf.data_ptr())
    assert e.value.status == B.EINVAL


def test_static_load_flow_rejects_five_scenarios():
    import torch
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import _binding as B
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    ibuf = torch.zeros(8, dtype=torch.int32, device="cuda")
    df = K.device_feeder(100, 5, ibuf.data_ptr(), ibuf.data_ptr(), buf.data_ptr(), buf.data_ptr(), np.zeros((3, 2)))
    with pytest.raises(K.OkrError) as e:
        K.power_flow_static(df, buf.data_ptr())
    assert e.value.status == B.EINVAL
