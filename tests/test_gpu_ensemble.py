"""Ensembles (tf_ensemble_*): groups of different grid sizes stepped by one
persistent cooperative launch over a ragged tile work-list.

Every site's arithmetic is the same whichever tile (and tile height) it falls
in, so an ensemble must reproduce, bit for bit, the same groups stepped one
context at a time; that is the oracle for this layer (the per-context path is
itself checked against the FP64 oracle in test_gpu_parity.py).
"""
import numpy as np
import pytest

from paper_2511_00445_gb300 import _binding as B

pytestmark = pytest.mark.gpu

FIELDS = (B.FIELD_PHI, B.FIELD_QXX, B.FIELD_QXY, B.FIELD_U1X, B.FIELD_U2Y, B.FIELD_F1 + 0,
          B.FIELD_F1 + 6, B.FIELD_F2 + 3, B.FIELD_F2 + 8)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_00445_gb300 import build
    build.build()


def groups_spec(storage=B.STORE_F32):
    """Three groups: ragged 40x36 (two instances), 64x48, and 33x17 whose
    rows are not 16-byte multiples (per-element tile loads)."""
    base = B.SolverParams(storage=storage)
    return [
        [base.with_(nx=40, ny=36, zeta=0.01), base.with_(nx=40, ny=36, zeta=0.002, lam=1.1)],
        [base.with_(nx=64, ny=48, zeta=0.005, K=0.08)],
        [base.with_(nx=33, ny=17, zeta=0.01, lam=0.3)],
    ]


def make_groups(spec):
    out = []
    for g, plist in enumerate(spec):
        tf = B.TwoFluid(plist)
        for b in range(len(plist)):
            tf.init_fields(seed=100 * g + b, phi0=0.5, dphi=0.01, S0=0.01)
        out.append(tf)
    return out


def alone(spec, steps):
    ref = make_groups(spec)
    for tf in ref:
        tf.step(steps)
        tf.sync()
    return ref


def assert_same(got, want):
    for g, (a, b) in enumerate(zip(got, want)):
        for inst in range(a.batch):
            for f in FIELDS:
                assert np.array_equal(a.read_field(inst, f), b.read_field(inst, f)), (g, inst, f)
        assert a.step_count() == b.step_count()


def test_ensemble_matches_groups_stepped_alone():
    spec = groups_spec()
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.step(1)          # LBM-only first pass
    ens.step(6)          # one persistent launch of six steps
    ens.sync()
    assert_same(grp, alone(spec, 7))
    cfg = ens.config()
    assert cfg["tile_y"] == 32 and cfg["ctas_per_sm"] == 2
    # 40x36: 2 x (2 x 2) tiles, 64x48: 2 x 2, 33x17: 2 x 1
    assert cfg["tiles_per_step"] == 8 + 4 + 2
    assert ens.launches() == 2


@pytest.mark.parametrize("nx,ny,storage", [(1024, 1024, B.STORE_F32), (1040, 1000, B.STORE_F32),
                                          (1030, 1000, B.STORE_F32), (1024, 1024, B.STORE_F16)])
def test_large_grid_matches_grid_stepped_alone(nx, ny, storage):
    """Grids of several waves of tiles: the persistent ensemble launch (its
    own tile numbering, populations read through L2 within the launch) and
    the per-context launches agree bit for bit, also with a ragged last tile
    column and row (1040 x 1000), rows that are not 16-byte multiples (1030:
    per-element tile loads) and 16-bit population storage."""
    spec = [[B.SolverParams(nx=nx, ny=ny, zeta=0.01, storage=storage)]]
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.step(1)
    ens.step(5)
    ens.sync()
    assert_same(grp, alone(spec, 6))


def test_ensemble_autotune_steps_are_real_steps():
    """Nine candidates (persistent launches with tile shapes 32x32, 32x24 and
    40x30 and one or two CTAs per SM; one launch per step with 32x32 or 40x30;
    the groups' own per-context launches) each run real steps; the trajectory
    equals stepping alone."""
    spec = groups_spec()
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.autotune(2)                       # first pass + 9 x 2 steps
    ens.step(3)
    ens.sync()
    assert_same(grp, alone(spec, 1 + 2 * B.ENS_CANDIDATES + 3))
    cfg = ens.config()
    assert len(cfg["us_per_step"]) == B.ENS_CANDIDATES == 9
    assert all(us > 0 for us in cfg["us_per_step"])
    assert cfg["tile_y"] in (0, 24, 30, 32) and cfg["ctas_per_sm"] in (1, 2)
    assert 0 <= cfg["candidate"] < 9
    assert cfg["persistent"] == (cfg["candidate"] < 6)


@pytest.mark.parametrize("candidate", [6, 7, 8])
@pytest.mark.parametrize("storage", [B.STORE_F32, B.STORE_BF16], ids=["f32", "bf16"])
def test_per_step_launch_candidates(candidate, storage):
    """Candidates 6 and 7 (one launch per step over every tile of every
    group, populations read through L1) and 8 (each group's own per-context
    launches) step the ragged groups bitwise like each context stepped alone,
    across a member read and repeated calls."""
    spec = groups_spec(storage)
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.select(candidate)
    l0 = ens.launches()
    ens.step(4)
    per_step = len(grp) if candidate == 8 else 1
    assert ens.launches() - l0 == 1 + 3 * per_step   # the LBM-only first pass, then the steps
    grp[1].read_field(0, B.FIELD_PHI)
    ens.step(3)
    ens.step(3)
    ens.sync()
    assert_same(grp, alone(spec, 10))
    cfg = ens.config()
    assert cfg["candidate"] == candidate and not cfg["persistent"]
    assert cfg["grid"] == cfg["tiles_per_step"] > 0
    with pytest.raises(B.TwoFluidError):
        ens.select(9)


@pytest.mark.parametrize("nx,ny,candidate", [(1040, 1000, 7), (1030, 1000, 6), (1024, 1024, 8)])
def test_per_step_launches_large_grid(nx, ny, candidate):
    """A grid of many waves of tiles, ragged last tile row and column (1040 x
    1000) and rows that are not 16-byte multiples (1030: per-element tile
    loads), through the per-step launches; 1024^2 through its own planned
    launches (the strip kernel)."""
    spec = [[B.SolverParams(nx=nx, ny=ny, zeta=0.01)]]
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.select(candidate)
    ens.step(6)
    ens.sync()
    assert_same(grp, alone(spec, 6))


def test_ensemble48_benchmarked_configuration():
    """The benchmarked ensemble: 48 instances of 128^2, 256^2 and 512^2 over
    the zeta / lambda / K combinations (instance b takes combination b mod 27
    of zeta in {0.001, 0.005, 0.01}, lambda in {0.3, 0.7, 1.1}, K in {0.02,
    0.04, 0.08}; seed b), autotuned (the launch shape it picks).  Every
    member equals the same instances stepped context by context, bit for bit,
    and the next step of a 512^2 member matches the FP64 oracle on windows."""
    from helpers import interior, oracle_params, read_state, window_step
    zetas, lams, ks = (0.001, 0.005, 0.01), (0.3, 0.7, 1.1), (0.02, 0.04, 0.08)
    spec = []
    for gi, n in enumerate((128, 256, 512)):
        spec.append([B.SolverParams(nx=n, ny=n, zeta=zetas[(b % 27) // 9], lam=lams[(b % 9) // 3],
                                    K=ks[b % 3]) for b in range(16 * gi, 16 * gi + 16)])

    def make():
        out = []
        for gi, plist in enumerate(spec):
            tf = B.TwoFluid(plist)
            for k in range(len(plist)):
                tf.init_fields(seed=16 * gi + k, phi0=0.5, dphi=0.01, S0=0.01, inst=k)
            out.append(tf)
        return out

    grp = make()
    ens = B.Ensemble(grp)
    ens.autotune(2)                       # first pass + 8 x 2 steps
    ens.step(5)
    ens.sync()
    ref = make()
    for tf in ref:
        tf.step(1 + 2 * B.ENS_CANDIDATES + 5)
        tf.sync()
    for g, (a, b) in enumerate(zip(grp, ref)):
        for inst in range(a.batch):
            for f in (B.FIELD_PHI, B.FIELD_QXY, B.FIELD_F1 + 5, B.FIELD_U2X):
                assert np.array_equal(a.read_field(inst, f), b.read_field(inst, f)), (g, inst, f)
    # one more ensemble step of a 512^2 member against the oracle on windows
    member, inst = grp[2], 7
    before = read_state(member, inst)
    op = oracle_params(spec[2][inst])
    ens.step(1)
    ens.sync()
    after = read_state(member, inst)
    H, WIN = 16, 32
    rng = np.random.default_rng(48)
    origins = [(0, 0), (512 - WIN // 2, 512 - WIN // 2)] + \
              [(int(rng.integers(0, 512)), int(rng.integers(0, 512))) for _ in range(3)]
    for x0, y0 in origins:
        ys, xs = (y0 + np.arange(WIN)) % 512, (x0 + np.arange(WIN)) % 512
        nxt, _ = window_step(before, op, x0, y0, WIN, WIN, H)
        for name in ("phi", "Qxx", "Qxy"):
            want = interior(getattr(nxt, name), H, WIN, WIN)
            got = getattr(after, name)[np.ix_(ys, xs)]
            spread = np.abs(getattr(before, name) - getattr(before, name).mean()).max()
            assert np.abs(got - want).max() <= 1e-6 * spread, (name, x0, y0)


def test_ensemble_member_reads_between_calls():
    """A member read completes that member's pending sub-steps; the next
    ensemble call realigns all members and the trajectory is unchanged."""
    spec = groups_spec()
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.step(3)
    grp[1].read_field(0, B.FIELD_PHI)
    ens.step(2)
    grp[0].conserved(1)
    ens.step(4)
    ens.sync()
    assert_same(grp, alone(spec, 9))


@pytest.mark.parametrize("storage", [B.STORE_F16, B.STORE_BF16], ids=["f16", "bf16"])
def test_ensemble_16bit_storage(storage):
    spec = groups_spec(storage)
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.step(5)
    ens.sync()
    assert_same(grp, alone(spec, 5))


def test_ensemble_repeated_calls_replay():
    """Equal calls reuse their launch shape; results stay identical."""
    spec = groups_spec()
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    for _ in range(4):
        ens.step(3)
    ens.sync()
    assert_same(grp, alone(spec, 12))
    assert ens.launches() == 1 + 4    # one first pass, then one launch per call


def test_ensemble_rejects_bad_members():
    base = B.SolverParams(nx=16, ny=16)
    a = B.TwoFluid(base)
    with pytest.raises(B.TwoFluidError):
        B.Ensemble([a, B.TwoFluid(base.with_(n_sub=3))])          # per-stage path only
    with pytest.raises(B.TwoFluidError):
        B.Ensemble([a, B.TwoFluid(base.with_(storage=B.STORE_F16))])
    with pytest.raises(B.TwoFluidError):
        B.Ensemble([a, a])


def test_grid_barrier_timeout_is_reported_and_recoverable():
    """Failure detection of the persistent launch without a device fault: with
    a short barrier poll limit and CTA 0 leaving at the first grid barrier
    without arriving, every other CTA's bounded wait runs out, the launch ends
    (tf_ensemble_sync returns, no hang) with TF_ERR_TIMEOUT, and afterwards the
    same ensemble steps freshly initialised members bitwise like per-context
    stepping."""
    spec = groups_spec()
    grp = make_groups(spec)
    ens = B.Ensemble(grp)
    ens.fault_drill(barrier_polls=1 << 12, held_cta=0)
    ens.step(4)                                  # LBM-only pass, then one launch of 3 steps
    with pytest.raises(B.TwoFluidError) as ei:
        ens.sync()
    assert ei.value.code == B.TF_ERR_TIMEOUT
    ens.sync()                                   # reported once, then clear
    ens.fault_drill(0, -1)
    for g, tf in enumerate(grp):
        for b in range(tf.batch):
            tf.init_fields(seed=100 * g + b, phi0=0.5, dphi=0.01, S0=0.01)
    ens.step(6)
    ens.sync()
    ens.close()
    assert_same(grp, alone(spec, 6))
