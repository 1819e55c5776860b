"""GPU: static and dynamic work-unit assignment of the streaming sweeps.

With dynamic assignment every CTA draws its next (tile, z-range) unit from a
global counter that the last CTA of each launch resets; results must not
depend on the assignment (each unit writes its own output points).  Checked:
bitwise equality over many consecutive launches (a counter left non-zero would
make a later launch skip units), with and without graphs, for batches and the
persistent launch, the plan report, the autotuner's candidates and argument
validation.  The every-variant tests of the sweep, temporal-blocking and
multi-field files run both assignments too.
"""
import json

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def heat(dims, so, sched, **kw):
    from paper_2404_02218_gb300.grid import Grid
    a = float(np.float32(0.8 * synthetic.heat_a_max(len(dims), so)))
    g = Grid(len(dims), dims, so, "heat", dt=a, **kw)
    g.set_schedule(sched)
    return g


@pytest.mark.parametrize("so", [2, 4, 8])
def test_many_launches_dynamic_equals_static(torch_cuda, so):
    dims = (200, 90, 37)
    u0 = synthetic.uniform_field(61, tuple(reversed(dims)))
    out = {}
    for sched in (0, 1):
        g = heat(dims, so, sched, temporal_block=1)
        assert json.loads(g.describe())["dyn"] == sched
        g.set_field("u", u0)
        for n in (1, 3, 7, 2):  # graphs of several lengths, replayed
            g.run(n)
        g.run(7)
        out[sched] = g.get_field("u")
        g.close()
    np.testing.assert_array_equal(out[1], out[0])


def test_dynamic_without_graphs_and_default(torch_cuda):
    dims = (150, 64, 30)
    u0 = synthetic.uniform_field(62, tuple(reversed(dims)))
    ref = heat(dims, 4, 0, temporal_block=1, use_graph=False)
    ref.set_field("u", u0)
    ref.run(11)
    for sched in (1, -1):
        g = heat(dims, 4, sched, temporal_block=1, use_graph=False)
        assert json.loads(g.describe())["dyn"] == 1  # the default is dynamic
        g.set_field("u", u0)
        for _ in range(11):
            g.run(1)
        np.testing.assert_array_equal(g.get_field("u"), ref.get_field("u"))


def test_batch_and_persistent(torch_cuda):
    from paper_2404_02218_gb300.grid import Batch
    cases = synthetic.batch_wave_cases(count=6, seed=15, lo=20, hi=48, so=4, nsteps=40)
    out = []
    for sched, persistent in ((0, False), (1, False), (1, True)):
        b = Batch(3, [dict(dims=c.dims, h=c.h, dt=c.dt) for c in cases], 4, "wave")
        b.set_schedule(sched)
        b.set_persistent(persistent)
        for i, c in enumerate(cases):
            b.set_field(i, "vel", c.velocity())
            b.set_source(i, c.src, c.f0, c.t0, c.amp)
        b.run(25)
        b.run(15)
        out.append([b.get_field(i, "u") for i in range(len(cases))])
        b.close()
    for got in out[1:]:
        for i in range(len(cases)):
            np.testing.assert_array_equal(got[i], out[0][i])


def test_tuner_tries_both_and_validation(torch_cuda):
    from paper_2404_02218_gb300 import native as N
    dims = (128, 64, 40)
    g = heat(dims, 8, -1, temporal_block=1)
    u0 = synthetic.uniform_field(63, tuple(reversed(dims)))
    g.set_field("u", u0)
    rep = g.tune(reps=1)
    assert {c["dyn"] for c in rep["candidates"]} == {0, 1}
    assert json.loads(g.describe())["dyn"] == rep["best"]["dyn"]
    np.testing.assert_array_equal(g.get_field("u"), u0)
    for bad in (2, -2):
        with pytest.raises(N.GbstError) as e:
            g.set_schedule(bad)
        assert e.value.status == N.GBST_EINVAL
