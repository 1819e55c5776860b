"""GPU parity: the CUDA sweeps against the FP64 oracle, element by element.

Tolerances (max-norm relative error, max |gpu - ref| / max |ref|, over the
interior at the final step): 1e-5 for FP32 storage, 2e-2 for BF16 storage.
Bitwise where the arithmetic is the same by construction: streaming vs simple
kernel, decomposed vs undecomposed, graph vs direct launches, checkpointed vs
uninterrupted runs.
"""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_grid(torch_cuda, *args, **kw):
    from paper_2404_02218_gb300.grid import Grid
    return Grid(*args, **kw)


def heat_case_run(torch_cuda, dims, so, nsteps, storage="f32", kernel="auto", decomp=(1, 1, 1), seed=5,
                  bc="zero", a=None, use_graph=True, tile=0):
    nd = len(dims)
    u0 = synthetic.uniform_field(seed, tuple(reversed(dims)))
    if a is None:
        a = float(np.float32(0.8 * synthetic.heat_a_max(nd, so)))
    g = make_grid(torch_cuda, nd, dims, so, "heat", storage=storage, h=1.0, dt=a, alpha=1.0, kernel=kernel,
                  decomp=decomp, bc=bc, use_graph=use_graph, tile=tile)
    g.set_field("u", u0)
    g.run(nsteps)
    out = g.get_field("u", np.float64)
    g.close()
    return u0, a, out


# ------------------------------------------------------------------ heat ---

def test_heat2d_256_gaussian_100_steps(torch_cuda):
    case = synthetic.heat2d_256()
    u0 = case.initial()
    g = make_grid(torch_cuda, 2, case.dims, case.so, "heat", h=1.0, dt=case.a, alpha=1.0)
    g.set_field("u", u0)
    g.run(case.nsteps)
    got = g.get_field("u")
    ref = oracle.heat_run(u0, case.so, case.a, case.nsteps)
    assert oracle.max_rel_error(got, ref) <= TOL_F32


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("dims", [(70, 45, 33), (129, 17, 9), (5, 3, 2), (1, 1, 1), (33, 66, 20)])
def test_heat3d_ragged(torch_cuda, so, dims):
    u0, a, got = heat_case_run(torch_cuda, dims, so, 7)
    ref = oracle.heat_run(u0, so, a, 7)
    assert oracle.max_rel_error(got, ref) <= TOL_F32


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("dims", [(300, 77), (8, 5), (1000, 3)])
def test_heat2d_ragged(torch_cuda, so, dims):
    u0, a, got = heat_case_run(torch_cuda, dims, so, 9)
    ref = oracle.heat_run(u0, so, a, 9)
    assert oracle.max_rel_error(got, ref) <= TOL_F32


@pytest.mark.parametrize("so", [2, 4, 8])
def test_heat_periodic_matches_oracle(torch_cuda, so):
    dims = (40, 36, 28)
    u0, a, got = heat_case_run(torch_cuda, dims, so, 11, bc="periodic")
    ref = oracle.heat_run(u0, so, a, 11, bc=oracle.BC_PERIODIC)
    assert oracle.max_rel_error(got, ref) <= TOL_F32


@pytest.mark.parametrize("so", [2, 4, 8])
def test_stream_kernel_equals_simple_kernel_bitwise(torch_cuda, so):
    dims = (90, 37, 21)
    _, _, a = heat_case_run(torch_cuda, dims, so, 5, kernel="stream")
    _, _, b = heat_case_run(torch_cuda, dims, so, 5, kernel="simple")
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("decomp", [(2, 2, 2), (3, 2, 1), (1, 1, 4)])
def test_decomposed_equals_undecomposed_bitwise(torch_cuda, so, decomp):
    dims = (68, 50, 44)
    _, _, ref = heat_case_run(torch_cuda, dims, so, 6)
    _, _, got = heat_case_run(torch_cuda, dims, so, 6, decomp=decomp)
    np.testing.assert_array_equal(got, ref)


def test_graph_equals_direct_bitwise(torch_cuda):
    dims = (50, 40, 30)
    _, _, a = heat_case_run(torch_cuda, dims, 4, 9, use_graph=True)
    _, _, b = heat_case_run(torch_cuda, dims, 4, 9, use_graph=False)
    np.testing.assert_array_equal(a, b)


def matching_variants(so, eq, storage, ndim):
    import json
    from paper_2404_02218_gb300 import native as N
    codes = {"heat": 0, "wave": 1, "f32": 0, "bf16": 1}
    out = []
    for i in range(N.stencil_variant_count()):
        v = json.loads(N.stencil_variant_info(i))
        if (v["R"], v["eq"], v["storage"], v["has_z"], v["nf"]) == (so // 2, codes[eq], codes[storage],
                                                                     int(ndim == 3), 1):
            out.append(i)
    return out


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("ndim", [3, 2])
def test_every_kernel_variant_bitwise(torch_cuda, so, storage, ndim):
    """Every compiled tile shape / depth / register variant gives the same bits as the simple kernel."""
    dims = (130, 70, 19) if ndim == 3 else (300, 77)
    u0 = synthetic.uniform_field(9, tuple(reversed(dims)))
    a = float(np.float32(0.8 * synthetic.heat_a_max(ndim, so)))
    ref = make_grid(torch_cuda, ndim, dims, so, "heat", storage=storage, dt=a, kernel="simple")
    ref.set_field("u", u0)
    ref.run(4)
    want = ref.get_field("u")
    variants = matching_variants(so, "heat", storage, ndim)
    assert variants
    g = make_grid(torch_cuda, ndim, dims, so, "heat", storage=storage, dt=a)
    for sched in (0, 1):  # static and dynamic work-unit assignment
        g.set_schedule(sched)
        for v in variants:
            for zc in (0, 3):
                g.set_field("u", u0)
                g.set_plan(v, 0, zc, 0)
                g.run(4)
                np.testing.assert_array_equal(g.get_field("u"), want,
                                              err_msg=f"variant {v} zchunks {zc} schedule {sched}")


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("ndim", [3, 2])
def test_every_wave_variant_bitwise(torch_cuda, so, storage, ndim):
    """Wave variants (kappa and u^{n-1} by TMA into the centre slots; 2D tiles and
    2D streamed along y) == the simple kernel, bit for bit."""
    dims = (130, 37, 21) if ndim == 3 else (300, 77)
    ref, *_ = wave_setup(torch_cuda, dims, so, storage=storage, kernel="simple")
    ref.run(5)
    want_u, want_p = ref.get_field("u"), ref.get_field("u_prev")
    variants = matching_variants(so, "wave", storage, ndim)
    assert variants
    for v in variants:
        for zc, sched in ((0, 1), (2, 1), (2, 0)):
            g, *_ = wave_setup(torch_cuda, dims, so, storage=storage)
            g.set_schedule(sched)
            g.set_plan(v, 0, zc, 0)
            g.run(5)
            msg = f"variant {v} zchunks {zc} schedule {sched}"
            np.testing.assert_array_equal(g.get_field("u"), want_u, err_msg=msg)
            np.testing.assert_array_equal(g.get_field("u_prev"), want_p, err_msg=msg)
            g.close()


def test_autotuner_keeps_fields_and_picks_a_plan(torch_cuda):
    import json
    dims = (96, 64, 48)
    g, *_ = wave_setup(torch_cuda, dims, 8)
    g.run(9)
    before_u, before_p = g.get_field("u"), g.get_field("u_prev")
    rep = g.tune(reps=2)
    assert rep["candidates"] and rep["best"]["variant"] in matching_variants(8, "wave", "f32", 3)
    np.testing.assert_array_equal(g.get_field("u"), before_u)
    np.testing.assert_array_equal(g.get_field("u_prev"), before_p)
    assert json.loads(g.describe())["variant"] == rep["best"]["variant"]


@pytest.mark.parametrize("so", [2, 8])
def test_heat_bf16_storage(torch_cuda, so):
    dims = (64, 48, 40)
    u0, a, got = heat_case_run(torch_cuda, dims, so, 10, storage="bf16")
    ref = oracle.heat_run(u0, so, a, 10)
    err = oracle.max_rel_error(got, ref)
    assert err <= TOL_BF16
    assert err > 0  # BF16 storage does round


# ------------------------------------------------------------------ wave ---

def wave_setup(torch_cuda, dims, so, storage="f32", decomp=(1, 1, 1), kernel="auto", seed=3, src=True,
               use_graph=True):
    nd = len(dims)
    h = 10.0
    speeds = synthetic.five_layer_speeds()
    c = synthetic.layered_velocity(tuple(reversed(dims)) if nd == 3 else (dims[1], dims[0]), speeds)
    dt = 0.5 * synthetic.wave_courant_max(nd, so) * h / max(speeds)
    g = make_grid(torch_cuda, nd, dims, so, "wave", storage=storage, h=h, dt=dt, decomp=decomp, kernel=kernel,
                  use_graph=use_graph)
    g.set_field("vel", c)
    pos = synthetic.source_position(seed, dims, margin=so)
    if src:
        g.set_source(pos, 10.0, 0.1, 1.0)
    return g, c, dt, h, pos


def wave_oracle(c, dt, h, so, nsteps, pos=None, uprev=None, u=None, step0=0, f0=10.0, t0=0.1, amp=1.0):
    kap = oracle.kappa_from_velocity(c, dt, h)
    shape = c.shape
    up = np.zeros(shape) if uprev is None else uprev
    uc = np.zeros(shape) if u is None else u
    return oracle.wave_run(up, uc, kap, so, nsteps, step0=step0, src=pos, f0=f0, t0=t0, amp=amp, dt=dt, h=h)


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("dims", [(48, 40, 36), (37, 29, 23)])
def test_wave3d_source_matches_oracle(torch_cuda, so, dims):
    n = 60
    g, c, dt, h, pos = wave_setup(torch_cuda, dims, so)
    g.run(n)
    got = g.get_field("u")
    gotp = g.get_field("u_prev")
    g.close()
    P, C = wave_oracle(c.astype(np.float64), dt, h, so, n, pos)
    assert np.max(np.abs(C)) > 0
    assert oracle.max_rel_error(got, C) <= TOL_F32
    assert oracle.max_rel_error(gotp, P) <= TOL_F32


@pytest.mark.parametrize("so", [2, 4, 8])
def test_wave2d_source_matches_oracle(torch_cuda, so):
    dims = (96, 80)
    n = 80
    g, c, dt, h, pos = wave_setup(torch_cuda, dims, so)
    g.run(n)
    got = g.get_field("u")
    g.close()
    _, C = wave_oracle(c.astype(np.float64), dt, h, so, n, pos)
    assert oracle.max_rel_error(got, C) <= TOL_F32


def test_wave_run_split_equals_single_run(torch_cuda):
    """run(13) + run(29) == run(42): source time and time-level rotation carry over."""
    dims = (40, 32, 28)
    g1, *_ = wave_setup(torch_cuda, dims, 4)
    g1.run(13)
    g1.run(29)
    a = g1.get_field("u")
    g2, *_ = wave_setup(torch_cuda, dims, 4)
    g2.run(42)
    b = g2.get_field("u")
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("so", [4, 8])
def test_wave_decomposed_equals_undecomposed_bitwise(torch_cuda, so):
    dims = (52, 44, 40)
    g1, *_ = wave_setup(torch_cuda, dims, so)
    g1.run(25)
    a = g1.get_field("u")
    g2, *_ = wave_setup(torch_cuda, dims, so, decomp=(2, 2, 2))
    g2.run(25)
    b = g2.get_field("u")
    np.testing.assert_array_equal(a, b)


def test_wave_checkpoint_resume_bitwise(torch_cuda):
    dims = (44, 36, 30)
    g1, *_ = wave_setup(torch_cuda, dims, 8)
    g1.run(30)
    ref = g1.get_field("u")
    g2, *_ = wave_setup(torch_cuda, dims, 8)
    g2.run(12)
    u = g2.get_field("u", np.float32)
    up = g2.get_field("u_prev", np.float32)
    step = g2.step
    g2.close()
    g3, *_ = wave_setup(torch_cuda, dims, 8)
    g3.set_field("u", u)
    g3.set_field("u_prev", up)
    g3.step = step
    g3.run(18)
    np.testing.assert_array_equal(g3.get_field("u"), ref)


@pytest.mark.parametrize("so", [4, 8])
def test_wave_bf16_storage(torch_cuda, so):
    dims = (48, 40, 36)
    n = 60
    g, c, dt, h, pos = wave_setup(torch_cuda, dims, so, storage="bf16")
    g.run(n)
    got = g.get_field("u")
    _, C = wave_oracle(c.astype(np.float64), dt, h, so, n, pos)
    assert oracle.max_rel_error(got, C) <= TOL_BF16


# ------------------------------------------------------------- reductions ---

@pytest.mark.parametrize("decomp", [(1, 1, 1), (2, 2, 2)])
def test_reductions_match_fp64_sums(torch_cuda, decomp):
    dims = (60, 50, 40)
    g, c, dt, h, pos = wave_setup(torch_cuda, dims, 4, decomp=decomp, src=False)
    u0 = synthetic.uniform_field(70, tuple(reversed(dims))) - np.float32(0.5)
    up = (0.9 * u0).astype(np.float32)
    g.set_field("u", u0)
    g.set_field("u_prev", up)
    g.run(7)
    u = g.get_field("u")
    v = g.get_field("u_prev")
    kap32 = g.get_field("vel").astype(np.float64)  # kappa as stored (FP32)
    assert g.reduce("sum") == pytest.approx(float(np.sum(u)), rel=1e-12, abs=1e-9)
    assert g.reduce("l2sq") == pytest.approx(float(np.sum(u * u)), rel=1e-12)
    assert g.reduce("maxabs") == float(np.max(np.abs(u)))
    e_ref = oracle.energy(u, v, kap32, 4)
    assert g.reduce("energy") == pytest.approx(e_ref, rel=1e-10)


def test_wave_energy_nearly_conserved_fp32(torch_cuda):
    dims = (64, 48, 40)
    g, *_ = wave_setup(torch_cuda, dims, 8, src=False)
    u0 = synthetic.uniform_field(71, tuple(reversed(dims))) - np.float32(0.5)
    g.set_field("u", u0)
    g.set_field("u_prev", u0)
    e0 = g.reduce("energy")
    g.run(200)
    e1 = g.reduce("energy")
    assert e0 > 0
    assert abs(e1 - e0) / e0 < 1e-4


# ---------------------------------------------------------------- errors ---

def test_unstable_heat_rejected(torch_cuda):
    from paper_2404_02218_gb300.native import GbstError, GBST_EUNSTABLE
    with pytest.raises(GbstError) as e:
        make_grid(torch_cuda, 3, (16, 16, 16), 4, "heat", dt=0.2, alpha=1.0, h=1.0)
    assert e.value.status == GBST_EUNSTABLE


def test_unstable_wave_velocity_rejected(torch_cuda):
    from paper_2404_02218_gb300.native import GbstError, GBST_EUNSTABLE
    dims = (16, 16, 16)
    g = make_grid(torch_cuda, 3, dims, 4, "wave", h=10.0, dt=0.01)
    with pytest.raises(GbstError) as e:
        g.set_field("vel", np.full((16, 16, 16), 4500.0, dtype=np.float32))
    assert e.value.status == GBST_EUNSTABLE
    with pytest.raises(GbstError):
        g.run(1)


def test_invalid_arguments(torch_cuda):
    from paper_2404_02218_gb300.native import GbstError, GBST_EINVAL
    with pytest.raises(GbstError) as e:
        make_grid(torch_cuda, 3, (16, 0, 16), 4, "heat", dt=0.01)
    assert e.value.status == GBST_EINVAL
    with pytest.raises(GbstError) as e:
        make_grid(torch_cuda, 3, (16, 16, 16), 6, "heat", dt=0.01)
    assert e.value.status == GBST_EINVAL
    g = make_grid(torch_cuda, 3, (16, 16, 16), 4, "heat", dt=0.01)
    with pytest.raises(GbstError) as e:
        g.set_field("u_prev", np.zeros((16, 16, 16), np.float32))
    assert e.value.status == GBST_EINVAL


def test_zero_and_negative_step_counts(torch_cuda):
    from paper_2404_02218_gb300.native import GbstError, GBST_EINVAL
    dims = (20, 12, 9)
    u0 = synthetic.uniform_field(40, tuple(reversed(dims)))
    g = make_grid(torch_cuda, 3, dims, 4, "heat", dt=0.05)
    g.set_field("u", u0)
    g.run(0)
    assert g.step == 0
    np.testing.assert_array_equal(g.get_field("u"), u0)
    with pytest.raises(GbstError) as e:
        g.run(-1)
    assert e.value.status == GBST_EINVAL


def test_plan_and_descriptor_validation(torch_cuda):
    import json
    from paper_2404_02218_gb300.native import GbstError, GBST_EINVAL
    with pytest.raises(GbstError) as e:
        make_grid(torch_cuda, 3, (16, 16, 16), 2, "heat", dt=0.05, temporal_block=3)
    assert e.value.status == GBST_EINVAL
    g = make_grid(torch_cuda, 3, (40, 30, 20), 2, "heat", dt=0.05)
    v = json.loads(g.describe())["variant"]
    with pytest.raises(GbstError) as e:
        g.set_plan(v, 7, 0, 0)  # a tile width the variant does not have
    assert e.value.status == GBST_EINVAL
    with pytest.raises(GbstError) as e:
        g.set_plan(10 ** 6, 0, 0, 0)
    assert e.value.status == GBST_EINVAL


@pytest.mark.parametrize("dims", [(1 << 20, 3, 2), (3, 1 << 16, 4), (4, 5, 1 << 16)])
@pytest.mark.parametrize("so", [4, 8])
def test_extreme_aspect_ratios(torch_cuda, dims, so):
    """One axis long (a million points in x; 65536 rows; 65536 planes, many z-chunks)."""
    u0, a, got = heat_case_run(torch_cuda, dims, so, 5)
    ref = oracle.heat_run(u0, so, a, 5)
    assert oracle.max_rel_error(got, ref) <= TOL_F32


@pytest.mark.parametrize("eq", ["heat", "wave"])
def test_wide_rows_layout(torch_cuda, eq):
    """Rows of at least 2 KB use 128-byte x ghosts (tensor maps shifted to the
    kernels' 16-byte halo): ragged wide grids, decomposed or not, match the
    simple kernel bit for bit and the oracle."""
    so = 8 if eq == "wave" else 4
    dims = (1030, 19, 11)
    if eq == "heat":
        u0 = synthetic.uniform_field(41, tuple(reversed(dims)))
        a = float(np.float32(0.8 * synthetic.heat_a_max(3, so)))
        outs = []
        for kw in (dict(kernel="simple"), {}, dict(decomp=(2, 1, 1))):
            g = make_grid(torch_cuda, 3, dims, so, "heat", h=1.0, dt=a, alpha=1.0, **kw)
            g.set_field("u", u0)
            g.run(5)
            outs.append(g.get_field("u", np.float64))
            g.close()
        for o in outs[1:]:
            np.testing.assert_array_equal(o, outs[0])
        assert oracle.max_rel_error(outs[1], oracle.heat_run(u0, so, a, 5)) <= TOL_F32
    else:
        ref, *_ = wave_setup(torch_cuda, dims, so, kernel="simple")
        ref.run(9)
        for kw in ({}, dict(decomp=(2, 1, 1))):
            g, *_ = wave_setup(torch_cuda, dims, so, **kw)
            g.run(9)
            np.testing.assert_array_equal(g.get_field("u"), ref.get_field("u"))
            np.testing.assert_array_equal(g.get_field("u_prev"), ref.get_field("u_prev"))
