"""GPU (sm_103a) path against the FP64 CPU oracle, through the C ABI.

FP64 storage must match the oracle to 1e-10 in the max norm relative to each
field's own max norm (rho, u, T) after a fixed number of steps; FP32
deviation storage must stay within 1e-4.  Lattices span several strips and
runs of rows with ragged tails, odd sizes, every wall orientation, both
extrapolation orders, moving walls, every EOS and viscosity law."""
import numpy as np
import pytest

from paper_1809_08683_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def lbm():
    from paper_1809_08683_gb300 import lbm as m
    m.build()
    m.load()
    return m


def rel(a, b, floor=1e-12):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def field_errors(mg, mo):
    # velocity errors relative to the max norm of the velocity vector field
    umax = max(np.hypot(mo["ux"], mo["uy"]).max(), 1e-12)
    return {"rho": rel(mg["rho"], mo["rho"]), "ux": np.abs(mg["ux"] - mo["ux"]).max() / umax,
            "uy": np.abs(mg["uy"] - mo["uy"]).max() / umax, "T": rel(mg["T"], mo["T"])}


TOLDEV32 = 1e-3


def dev_errors(mg, mo, rho0=1.0, T0=1.0):
    """Errors of the deviations rho - rho0 and T - T0, each relative to its
    own max norm.  Where a flow's density and temperature vary little (the
    heating of a channel flow is 1e-4 of T0), a tolerance relative to the
    field itself would admit large errors in the variation."""
    return {"rho_dev": rel(mg["rho"] - rho0, mo["rho"] - rho0), "T_dev": rel(mg["T"] - T0, mo["T"] - T0)}


def pair(orc, lbm, cfg, steps, seed=None, df=0.0, tile=None):
    o = orc.Oracle(cfg, threads=8)
    g = lbm.Lattice(cfg)
    if tile:
        g.set_tile(*tile)
    if seed is not None:
        rho, ux, uy, T = W.random_macros(cfg["nx"], cfg["ny"], seed)
        o.init_macros(rho, ux, uy, T)
        g.init_macros(rho, ux, uy, T)
        if df:
            nf, ng = W.df_noise(cfg["nx"], cfg["ny"], seed + 1, df)
            fo, go = o.get_state()
            o.set_state(fo + nf, go + ng)
            fg, gg = g.get_state()
            g.set_state(fg + nf, gg + ng)
    assert o.step(steps) == 0
    g.step(steps)
    return o, g, field_errors(g.macros(), o.macros())


def assert_close(err, tol):
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, (bad, err)


@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 4), (1, 8), (16, 16)])
def test_periodic_small_fp64(orc, lbm, nx, ny):
    cfg = W.periodic_box(nx, ny, visc_law=2, eos=(W.EOS_CUBIC, (0.05, 0.2)), gamma=1.3,
                         force=(1e-5, -2e-5))
    _, _, err = pair(orc, lbm, cfg, 1000, seed=nx * 100 + ny, df=1e-4)
    assert_close(err, TOL64)


@pytest.mark.parametrize("bx,by", [(32, 1), (32, 37), (64, 1), (64, 5), (128, 37), (128, 4)])
def test_periodic_multitile_ragged_fp64(orc, lbm, bx, by):
    cfg = W.periodic_box(200, 37, visc_law=1, eos=(W.EOS_IDEAL, ()), force=(2e-5, 0.0))
    _, _, err = pair(orc, lbm, cfg, 60, seed=17, df=1e-4, tile=(bx, by))
    assert_close(err, TOL64)


@pytest.mark.parametrize("eos,gamma", [((W.EOS_DECOUPLING, ()), 1.4), ((W.EOS_CS, ()), 1.1),
                                       ((W.EOS_IDEAL, ()), 1.4), ((W.EOS_CUBIC, (0.05, 0.2)), 1.3)])
def test_every_eos_fp64(orc, lbm, eos, gamma):
    cfg = W.periodic_box(24, 10, eos=eos, gamma=gamma, visc_law=2)
    _, _, err = pair(orc, lbm, cfg, 300, seed=23, df=1e-4)
    assert_close(err, TOL64)


def test_corrections_off_fp64(orc, lbm):
    cfg = W.periodic_box(24, 10, corrections=0)
    _, _, err = pair(orc, lbm, cfg, 300, seed=29, df=1e-4)
    assert_close(err, TOL64)


def test_couette_4x64_fp64(orc, lbm):
    # 4 x 64, lid 0.05, both walls at T = 1, ideal gas, Pr 0.71, tau 0.8, 20000 steps
    _, _, err = pair(orc, lbm, W.couette(nx=4, ny=64), 20000)
    assert_close(err, TOL64)


def test_poiseuille_4x128_cubic_fp64(orc, lbm):
    # 4 x 128, cubic EOS a = 0.05, b = 0.2, gamma 1.3, Pr 0.7, 50000 steps
    _, _, err = pair(orc, lbm, W.poiseuille(nx=4, ny=128), 50000)
    assert_close(err, TOL64)


@pytest.mark.parametrize("tile", [None, (32, 16), (64, 3), (128, 64)])
def test_cavity_fp64(orc, lbm, tile):
    cfg = W.cavity(N=64, Ra=1e3, eps=0.6)
    _, _, err = pair(orc, lbm, cfg, 1000, tile=tile)
    assert_close(err, TOL64)


@pytest.mark.parametrize("order", [1, 2])
def test_cavity_ragged_moving_lid_fp64(orc, lbm, order):
    cfg = W.cavity(N=33, Ra=300.0, eps=0.4, tau0=0.7, order=order)
    cfg["nx"] = 150
    cfg["walls"][1]["u"] = (0.03, 0.0)
    _, _, err = pair(orc, lbm, cfg, 200, seed=31, df=1e-4, tile=(128, 7))
    assert_close(err, TOL64)


def test_x_walls_y_periodic_fp64(orc, lbm):
    cfg = W.periodic_box(23, 9)
    cfg["walls"][2] = W.wall((0.0, 0.02), 1.1, 0, 2)
    cfg["walls"][3] = W.wall((0.0, 0.0), 0.9, 1, 1)
    _, _, err = pair(orc, lbm, cfg, 300, seed=37, df=1e-4)
    assert_close(err, TOL64)


def test_minimal_walled_lattice_fp64(orc, lbm):
    cfg = W.cavity(N=4, Ra=10.0, eps=0.2, tau0=0.8)
    _, _, err = pair(orc, lbm, cfg, 200)
    assert_close(err, TOL64)


def test_cavity_512_bench_shape_fp64(orc, lbm):
    # full-size configuration (512^2, Ra 1e6) in the default launch shape
    cfg = W.cavity(N=512, Ra=1e6, eps=0.6)
    _, _, err = pair(orc, lbm, cfg, 20)
    assert_close(err, TOL64)


def test_poiseuille_4x128_cubic_fp32(orc, lbm):
    cfg = W.poiseuille(nx=4, ny=128, precision=1)
    o, g, err = pair(orc, lbm, cfg, 50000)
    assert_close(err, TOL32)
    # the heating T - T0 itself (max 4.5e-4) and the density variation are
    # resolved to 1e-3 of their own size
    assert_close(dev_errors(g.macros(), o.macros()), TOLDEV32)


@pytest.mark.parametrize("bx,by,pr", [(64, 5, 1), (128, 64, 1), (256, 16, 1), (128, 9, 2), (256, 32, 2),
                                      (32, 7, 3), (128, 32, 3)])
def test_paired_fp32_periodic_ragged(orc, lbm, bx, by, pr):
    # odd width: the last pair of the last strip has one node only
    cfg = W.periodic_box(201, 37, visc_law=2, eos=(W.EOS_CUBIC, (0.05, 0.2)), gamma=1.3,
                         force=(2e-5, -1e-5), precision=1)
    _, _, err = pair(orc, lbm, cfg, 100, seed=41, df=1e-4, tile=(bx, by, pr))
    assert_close(err, TOL32)


@pytest.mark.parametrize("N,tile", [(67, (128, 16, 1)), (67, (64, 7, 1)), (67, (256, 16, 2)),
                                    # east wall in a last strip of 1 or 2 columns: the node two
                                    # columns inward lies beyond the strip's left halo, or in it
                                    (65, (64, 7, 1)), (66, (64, 7, 1))])
def test_paired_fp32_walls(orc, lbm, N, tile):
    cfg = W.cavity(N=N, Ra=1e3, eps=0.6, precision=1)
    cfg["walls"][1]["u"] = (0.02, 0.0)
    o, g, err = pair(orc, lbm, cfg, 1500, tile=tile)
    assert_close(err, TOL32)
    assert abs(g.nusselt(W.WALL_W) / o.nusselt(W.WALL_W) - 1) < 5e-3


def test_paired_fp32_poiseuille_4x128_cubic(orc, lbm):
    cfg = W.poiseuille(nx=4, ny=128, precision=1)
    o, g, err = pair(orc, lbm, cfg, 50000, tile=(64, 32, 2))
    assert_close(err, TOL32)
    assert_close(dev_errors(g.macros(), o.macros()), TOLDEV32)


def test_paired_fp64_rejected(lbm):
    g = lbm.Lattice(W.periodic_box(16, 8))
    for pr in (1, 2, 3):
        assert g.L.lbm_set_tile(g.h, 128, 8, pr) == lbm.LBM_EINVAL
    assert g.L.lbm_set_tile(g.h, 120, 8, 5) == lbm.LBM_EINVAL


@pytest.mark.parametrize("bx,by", [(60, 1), (60, 7), (120, 37), (240, 16)])
def test_paired_warp_strips_periodic_ragged(orc, lbm, bx, by):
    # 201 columns: the last pair is half filled and holds the wrapped column 0
    cfg = W.periodic_box(201, 37, visc_law=2, eos=(W.EOS_CUBIC, (0.05, 0.2)), gamma=1.3,
                         force=(2e-5, -1e-5), precision=1)
    _, _, err = pair(orc, lbm, cfg, 100, seed=47, df=1e-4, tile=(bx, by, 5))
    assert_close(err, TOL32)


@pytest.mark.parametrize("nx,ny", [(3, 3), (1, 8), (61, 5), (64, 4)])
def test_paired_warp_strips_small_periodic(orc, lbm, nx, ny):
    cfg = W.periodic_box(nx, ny, visc_law=2, eos=(W.EOS_IDEAL, ()), force=(1e-5, -2e-5), precision=1)
    _, _, err = pair(orc, lbm, cfg, 300, seed=nx * 100 + ny, df=1e-4, tile=(60, 2, 5))
    assert_close(err, TOL32)


@pytest.mark.parametrize("tile", [(60, 16, 5), (120, 7, 5)])
def test_paired_warp_strips_walls(orc, lbm, tile):
    # odd side: the east wall column is the first node of a pair
    cfg = W.cavity(N=67, Ra=1e3, eps=0.6, precision=1)
    cfg["walls"][1]["u"] = (0.02, 0.0)
    o, g, err = pair(orc, lbm, cfg, 1500, tile=tile)
    assert_close(err, TOL32)
    assert abs(g.nusselt(W.WALL_W) / o.nusselt(W.WALL_W) - 1) < 5e-3


def test_paired_warp_strips_even_walls(orc, lbm):
    # even side: the east wall column is the second node of a pair
    cfg = W.cavity(N=64, Ra=1e3, eps=0.6, precision=1)
    _, _, err = pair(orc, lbm, cfg, 1500, tile=(60, 9, 5))
    assert_close(err, TOL32)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("bx,by", [(30, 1), (60, 5), (120, 37), (120, 4)])
def test_warp_strips_periodic_ragged(orc, lbm, precision, bx, by):
    # 200 columns: the last warp strip is 20 columns wide, the last CTA ragged
    cfg = W.periodic_box(200, 37, visc_law=2, eos=(W.EOS_CUBIC, (0.05, 0.2)), gamma=1.3,
                         force=(2e-5, -1e-5), precision=precision)
    _, _, err = pair(orc, lbm, cfg, 60, seed=43, df=1e-4, tile=(bx, by, 4))
    assert_close(err, TOL32 if precision else TOL64)


@pytest.mark.parametrize("nx,ny", [(3, 3), (1, 8), (31, 5), (32, 4)])
def test_warp_strips_small_periodic_fp64(orc, lbm, nx, ny):
    # both wrap chunks in one warp; a strip narrower than the warp
    cfg = W.periodic_box(nx, ny, visc_law=2, eos=(W.EOS_IDEAL, ()), force=(1e-5, -2e-5))
    _, _, err = pair(orc, lbm, cfg, 300, seed=nx * 100 + ny, df=1e-4, tile=(120, 2, 4))
    assert_close(err, TOL64)


@pytest.mark.parametrize("tile", [(120, 16, 4), (30, 7, 4)])
def test_warp_strips_walls_fp64(orc, lbm, tile):
    cfg = W.cavity(N=67, Ra=1e3, eps=0.6, tau0=0.8)
    cfg["walls"][1]["u"] = (0.02, 0.0)
    o, g, err = pair(orc, lbm, cfg, 1000, tile=tile)
    assert_close(err, TOL64)
    assert abs(g.nusselt(W.WALL_W) / o.nusselt(W.WALL_W) - 1) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_warp_strips_equal_block_strips(lbm, precision):
    # the warp-strip kernel runs the per-node arithmetic of the block-strip
    # kernel on the same inputs: the two give the same bits
    cfg = W.cavity(N=197, Ra=2e3, eps=0.5, precision=precision)
    a, b = lbm.Lattice(cfg), lbm.Lattice(cfg)
    a.set_tile(128, 16, 0)  # both shapes run the instance specialised for the cavity model
    b.set_tile(30, 11, 4)
    a.step(300)
    b.step(300)
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


@pytest.mark.parametrize("eos", [(W.EOS_IDEAL, ()), (W.EOS_CUBIC, (0.05, 0.2))])
def test_cavity_model_instance_fp64(orc, lbm, eos):
    # the default shape runs the kernel instance specialised for the cavity
    # model (Sutherland, F = rho g, corrections; ideal or cubic EOS)
    cfg = W.cavity(N=190, Ra=2e3, eps=0.5, eos=eos, gamma=1.3 if eos[0] == W.EOS_CUBIC else 1.4)
    _, _, err = pair(orc, lbm, cfg, 300)
    assert_close(err, TOL64)


@pytest.mark.parametrize("eos", [(W.EOS_IDEAL, ()), (W.EOS_CUBIC, (0.05, 0.2))])
def test_cavity_model_instance_vs_generic_fp32(lbm, eos):
    # pair 3 (macros recomputed at collision time) runs the generic instance
    cfg = W.cavity(N=190, Ra=2e3, eps=0.5, eos=eos, gamma=1.3 if eos[0] == W.EOS_CUBIC else 1.4, precision=1)
    g, h = lbm.Lattice(cfg), lbm.Lattice(cfg)
    h.set_tile(64, 9, 3)
    g.step(800)
    h.step(800)
    mg, mh = g.macros(), h.macros()
    umax = np.hypot(mg["ux"], mg["uy"]).max()
    assert rel(mh["rho"], mg["rho"]) < 1e-5 and rel(mh["T"], mg["T"]) < 1e-5
    assert np.abs(mh["ux"] - mg["ux"]).max() / umax < 1e-4


@pytest.mark.parametrize("N,tile", [(190, (128, 12, 1)), (194, (64, 7, 1))])
@pytest.mark.parametrize("eos", [(W.EOS_IDEAL, ()), (W.EOS_CUBIC, (0.05, 0.2))])
def test_cavity_model_instance_paired_fp32(orc, lbm, N, tile, eos):
    # paired block strips run the cavity instance too (N^2 >= 32768 nodes);
    # 194 columns in strips of 64 leave a last strip of 2 columns
    cfg = W.cavity(N=N, Ra=2e3, eps=0.5, eos=eos, gamma=1.3 if eos[0] == W.EOS_CUBIC else 1.4, precision=1)
    o, g, err = pair(orc, lbm, cfg, 300, seed=N, df=1e-4, tile=tile)
    assert_close(err, TOL32)


def test_model_classes_batched_equal_alone(lbm):
    # a cavity of 64^2 nodes runs the generic instance, one of 200^2 the
    # cavity instance; a batch launches them as two groups: every member
    # steps as it would alone
    import torch
    stream = torch.cuda.Stream()
    cfgs = [W.cavity(N=64, Ra=1e3, eps=0.3, precision=1), W.cavity(N=200, Ra=1e4, eps=0.3, precision=1),
            W.couette(nx=40, ny=12, precision=1)]
    alone = [lbm.Lattice(c, stream=stream) for c in cfgs]
    mixed = [lbm.Lattice(c, stream=stream) for c in cfgs]
    b = lbm.Batch(mixed, graph_steps=0)
    b.step(30)
    for a in alone:
        a.step(30)
    stream.synchronize()
    for a, m in zip(alone, mixed):
        fa, ga = a.get_state()
        fm, gm = m.get_state()
        assert np.array_equal(fa, fm) and np.array_equal(ga, gm)
    b.close()


def test_batch_rejects_changed_eos_class(lbm):
    import torch
    stream = torch.cuda.Stream()
    cfg = W.cavity(N=200, Ra=1e3, eps=0.3)  # large enough for the cavity instance
    lat = lbm.Lattice(cfg, stream=stream)
    b = lbm.Batch([lat], graph_steps=0)
    b.step(2)
    lat.check(lat.L.lbm_set_eos(lat.h, W.EOS_DECOUPLING, None, 0))
    with pytest.raises(Exception):
        b.step(2)
    b.close()


def test_lean_one_node_shape_matches_oracle(orc, lbm):
    # pair 3 recomputes the macros at collision time; the compiler may contract
    # that second copy differently, so it agrees with pair 0 to FP32 rounding
    cfg = W.cavity(N=70, Ra=2e3, eps=0.5, precision=1)
    _, _, err = pair(orc, lbm, cfg, 1500, tile=(64, 9, 3))
    assert_close(err, TOL32)


def test_couette_4x64_fp32(orc, lbm):
    cfg = W.couette(nx=4, ny=64, precision=1)
    o, g, err = pair(orc, lbm, cfg, 20000)
    assert_close(err, TOL32)
    # the viscous heating T - T0 peaks at 1.9e-4: checked against its own size
    assert_close(dev_errors(g.macros(), o.macros()), TOLDEV32)


def test_cavity_fp32(orc, lbm):
    cfg = W.cavity(N=64, Ra=1e3, eps=0.6, precision=1)
    o, g, err = pair(orc, lbm, cfg, 2000)
    assert_close(err, TOL32)
    assert abs(g.nusselt(W.WALL_W) / o.nusselt(W.WALL_W) - 1) < 5e-3


def test_nusselt_and_diagnostics_fp64(orc, lbm):
    cfg = W.cavity(N=48, Ra=1e3, eps=0.6, tau0=0.8)
    o, g, err = pair(orc, lbm, cfg, 1500)
    assert_close(err, TOL64)
    for wall in (W.WALL_W, W.WALL_E):
        assert abs(g.nusselt(wall) / o.nusselt(wall) - 1) < 1e-10
    mo = o.macros()
    d = g.diagnostics()
    assert abs(d["mass"] / mo["rho"].sum() - 1) < 1e-13
    w = np.ones(48)
    w[0] = w[-1] = 0.5
    pstar = (w[:, None] * w[None, :] * mo["p"]).sum() / (47.0 ** 2) / o.derived()["p0"]
    assert abs(d["pstar"] / pstar - 1) < 1e-12
    assert d["nonfinite"] == 0


def test_mass_conservation_and_residual(lbm):
    cfg = W.cavity(N=40, Ra=1e3, eps=0.5, tau0=0.8)
    g = lbm.Lattice(cfg)
    d0 = g.diagnostics(snapshot=True)
    m0 = g.macros()
    g.step(500)
    m1 = g.macros()
    d1 = g.diagnostics(snapshot=True)
    assert abs(d1["mass"] / d0["mass"] - 1) < 1e-13
    du = np.sqrt(((m1["ux"] - m0["ux"]) ** 2 + (m1["uy"] - m0["uy"]) ** 2).sum()
                 / (m1["ux"] ** 2 + m1["uy"] ** 2).sum())
    dT = np.sqrt(((m1["T"] - m0["T"]) ** 2).sum() / ((m1["T"] - 1.0) ** 2).sum())
    assert abs(d1["residual"] / max(du, dT) - 1) < 1e-10


def test_nan_injection_reports_unstable(lbm):
    cfg = W.periodic_box(16, 8)
    g = lbm.Lattice(cfg)
    f, gg = g.get_state()
    f[2, 3, 4] = np.nan
    g.set_state(f, gg)
    assert g.status_step(3) == lbm.LBM_EUNSTABLE
    assert g.L.lbm_step(g.h, 1) == lbm.LBM_EUNSTABLE  # sticky
    eos = cfg["eos"]
    g.check(g.L.lbm_set_eos(g.h, eos["kind"], None, 0))  # re-initialisation clears it
    assert g.status_step(3) == lbm.LBM_OK


def _mixed_lattices(lbm):
    cfgs = [W.cavity(N=40, Ra=1e3, eps=0.6, tau0=0.7),
            W.cavity(N=70, Ra=2e3, eps=0.3, eos=(W.EOS_CUBIC, (0.05, 0.2)), precision=1),
            W.poiseuille(nx=5, ny=33),
            W.couette(nx=130, ny=12, precision=1)]
    return cfgs


@pytest.mark.parametrize("graph_steps", [0, 10])
def test_batch_equals_alone(lbm, graph_steps):
    import torch
    stream = torch.cuda.Stream()
    cfgs = _mixed_lattices(lbm)
    alone = [lbm.Lattice(c, stream=stream) for c in cfgs]
    mixed = [lbm.Lattice(c, stream=stream) for c in cfgs]
    alone[1].set_tile(64, 9)
    mixed[1].set_tile(64, 9)
    alone[3].set_tile(64, 5, 1)
    mixed[3].set_tile(64, 5, 1)
    for a in alone[:2]:
        a.step(7)        # odd step count: the batch must respect each lattice's parity
    for m in mixed[:2]:
        m.step(7)
    b = lbm.Batch(mixed, graph_steps=graph_steps)
    b.step(20)
    for a in alone[:2]:
        a.step(20)
    for a in alone[2:]:
        a.step(20)
    stream.synchronize()
    for a, m in zip(alone, mixed):
        fa, ga = a.get_state()
        fm, gm = m.get_state()
        assert a.steps == m.steps
        assert np.array_equal(fa, fm) and np.array_equal(ga, gm)
    b.close()


def test_couette_variable_viscosity_parity(orc, lbm):
    # Sec. 4.2 with mu / mu0 = T / T0: adiabatic (Neumann) lower wall at rest,
    # Dirichlet lid at U0 = 0.108, second-order extrapolation; the start-up
    # transient against the oracle.  FP64 at Pr = 20; FP32 at Pr = 0.71: at
    # Pr = 20 the model's grid-scale modes across x are unstable (pinned on
    # the oracle), and the x-dependent stochastic rounding of FP32 storage
    # excites them, while the x-invariant FP64 flow never does.
    for precision, tol, Pr in ((0, TOL64, 20.0), (1, TOL32, 0.71)):
        cfg = W.couette_variable_mu(nx=4, ny=32, Ma_e=0.1, Pr=Pr, precision=precision)
        o, g, err = pair(orc, lbm, cfg, 3000)
        assert_close(err, tol)
        assert_close(dev_errors(g.macros(), o.macros()), 1e-8 if precision == 0 else TOLDEV32)


@pytest.mark.parametrize("precision,Pr,eos", [(0, 20.0, (W.EOS_IDEAL, ())), (0, 20.0, (W.EOS_DECOUPLING, ())),
                                             (1, 0.71, (W.EOS_IDEAL, ()))])
def test_couette_variable_viscosity_closed_form(lbm, precision, Pr, eos):
    # steady state against Eq. Couette.u.T at Ma_e = 0.1; the paper finds u
    # and T the same for every EOS.  Pr = 20 (FP64): 10% heating at the
    # adiabatic wall, and u 1.6% away from the linear profile of constant
    # viscosity; the oracle's steady state is 1.1e-3 (u) and 3.1e-3 (T - T0)
    # from the closed form (ideal gas), 1.0e-3 and 2.7e-3 (decoupling).
    # Pr = 0.71 (FP32): the oracle is 1.0e-3 and 2.7e-3 away.
    import torch
    from closed_forms import couette_mu_profile
    ny = 32
    cfg = W.couette_variable_mu(nx=4, ny=ny, Ma_e=0.1, Pr=Pr, eos=eos, precision=precision)
    lat = lbm.Lattice(cfg, stream=torch.cuda.Stream())
    batch = lbm.Batch([lat], graph_steps=10000)
    batch.step(600000 if Pr > 1 else 100000)
    m = lat.macros()
    batch.close()
    U0 = cfg["walls"][1]["u"][0]
    Ma = U0 / np.sqrt(lat.derived()["Cp"])
    xi = np.arange(ny) / (ny - 1.0)
    s, Ta = couette_mu_profile(xi, Ma, Pr)
    for col in range(4):
        ux, T = m["ux"][:, col] / U0, m["T"][:, col]
        eu = np.sqrt(((ux - s) ** 2).sum() / (s ** 2).sum())
        eT = np.sqrt(((T - Ta) ** 2).sum() / ((Ta - 1.0) ** 2).sum())
        assert eu < 2e-3 and eT < 6e-3, (col, eu, eT)
        if Pr > 1:
            # constant viscosity would give u = U0 xi, far from this result
            assert np.sqrt(((ux - xi) ** 2).sum() / (xi ** 2).sum()) > 5 * eu

