"""Phase-batched fits (mpm_fit_batch with opts.graph = 2).

Subjects that share the map count, the preconditioner and the echo storage
run as one batch class: every phase of every Newton update (JTV reweighting,
voxel pass, PCG start, each PCG iteration, PCG end, posterior variance) is
one kernel launch for up to 16 subjects, each subject on its own share of the
blocks with its own CG scalars.  The iteration kernel's wave of blocks is
split between the subjects, so a subject's reductions run over fewer blocks
than in its solo fit and sum in another order: each subject must match its
solo fit within the fit tolerances (objective 1e-5 relative at every
update, maps 1e-3 in map units, posterior variance 5e-3 relative), and two
subjects must match the FP64 oracle's fit.  The launch count checks that a
group really takes one launch per phase.
"""
import numpy as np
import pytest

import oracle as orc
from cases import dataset, map_error, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


# shape, seed, contrasts, echoes, bfloat16 echoes, with a variance output.
# The staged iteration takes x sizes that are multiples of 4, with the tile's
# box inside the volume: 32 x 8 tiles from x >= 40 (and y >= 10), 16 x 16
# below (x >= 24, y >= 18).
SUBJECTS = [
    ((48, 40, 20), 101, ("PDw", "T1w", "MTw"), (8, 8, 6), False, True),       # K4 32x8
    ((36, 20, 9), 102, ("PDw", "T1w"), (6, 4), False, True),                  # K3 16x16
    ((64, 24, 12), 103, ("PDw", "T1w", "MTw"), (5, 7, 4), True, True),        # K4 bf16 32x8
    ((28, 20, 20), 104, ("PDw", "T1w", "MTw", "VFA15"), (4, 4, 4, 4), False, True),  # K4 16x16
    ((40, 28, 13), 105, ("PDw", "T1w", "MTw"), (6, 6, 5), False, False),      # K4 32x8
    ((44, 36, 10), 106, ("PDw", "T1w"), (5, 5), False, False),                # K3 32x8
    ((32, 18, 11), 107, ("PDw", "T1w", "MTw"), (4, 5, 3), False, False),      # K4 16x16
]
INIT_LAUNCHES = 3       # per subject: image means (two kernels) and the constant maps


def _subject(mpm, spec):
    import torch
    shape, seed, contrasts, echoes, bf16, with_var = spec
    d = dataset(shape, seed=seed, contrasts=contrasts, n_echoes=echoes)
    pg = mpm.make_problem(d["prot"], shape, echo_dtype=1 if bf16 else 0)
    x = to_dev(d["x"])
    if bf16:
        x = x.to(torch.bfloat16)
        d["x"] = x.float().cpu().numpy()
    return d, pg, x, with_var


def _zeros(pg, d):
    import torch
    return torch.zeros((pg.n_maps, int(np.prod(d["shape"]))), dtype=torch.float32, device="cuda")


def _solo(mpm, d, pg, x, with_var, opts):
    y = _zeros(pg, d)
    var = _zeros(pg, d) if with_var else None
    st, rep = mpm.mpm_fit(pg, opts, x, y, to_dev(d["b1p"]), to_dev(d["b1m"]), var=var)
    return y, var, rep


def _batch(mpm, subs, opts):
    ys = [_zeros(pg, d) for d, pg, _, _ in subs]
    vs = [_zeros(pg, d) if v else None for d, pg, _, v in subs]
    before = mpm.mpm_kernel_launches()
    st, reps = mpm.mpm_fit_batch([pg for _, pg, _, _ in subs], opts, [x for _, _, x, _ in subs], ys,
                                 b1ps=[to_dev(d["b1p"]) for d, _, _, _ in subs],
                                 b1ms=[to_dev(d["b1m"]) for d, _, _, _ in subs], vars=vs)
    return ys, vs, reps, mpm.mpm_kernel_launches() - before


def _launches_per_group(gn, cg, with_var):
    # JTV + voxel pass at each of gn + 1 evaluations, PCG start + cg iterations
    # + PCG end per update, the variance (its JTV weights are the last fresh
    # ones when they are refreshed at every update)
    return 2 * (gn + 1) + gn * (cg + 2) + (1 if with_var else 0)


def _check_equal_to_solo(sol, yb, vb, rb, gn, tag):
    y, var, rep = sol
    assert rb.iters == rep.iters == gn, tag
    np.testing.assert_allclose(np.array(rb.F[:gn + 1]), np.array(rep.F[:gn + 1]), rtol=1e-5,
                               err_msg=str(tag))
    assert map_error(to_np(yb), to_np(y)).max() <= 1e-3, tag
    if var is not None:
        np.testing.assert_allclose(to_np(vb), to_np(var), rtol=5e-3, err_msg=str(tag))


def test_phased_batch_matches_solo_fits(mpm):
    gn, cg = 6, 30
    subs = [_subject(mpm, s) for s in SUBJECTS]
    solos = [_solo(mpm, d, pg, x, v, mpm.make_opts(gn_iters=gn, cg_iters=cg)) for d, pg, x, v in subs]
    ys, vs, reps, launches = _batch(mpm, subs, mpm.make_opts(gn_iters=gn, cg_iters=cg, graph="phased"))
    for i, (sol, yb, vb, rb) in enumerate(zip(solos, ys, vs, reps)):
        _check_equal_to_solo(sol, yb, vb, rb, gn, i)
    # five classes: K = 4 float32 32x8 (subjects 0, 4) and 16x16 (3, 6),
    # K = 3 float32 16x16 (1) and 32x8 (5), K = 4 bfloat16 32x8 (2); all but
    # the one of subject 5 have a variance output
    expect = 4 * _launches_per_group(gn, cg, True) + _launches_per_group(gn, cg, False)
    assert launches == expect + INIT_LAUNCHES * len(subs), launches


def test_phased_replay_is_bit_identical(mpm):
    subs = [_subject(mpm, s) for s in SUBJECTS[:2]]
    opts = mpm.make_opts(gn_iters=3, cg_iters=20, graph="phased")
    first = _batch(mpm, subs, opts)
    again = _batch(mpm, subs, opts)        # the cached graph
    for a, b in zip(first[0], again[0]):
        assert np.array_equal(to_np(a), to_np(b))
    for a, b in zip(first[2], again[2]):
        assert list(a.F[:4]) == list(b.F[:4])
    assert first[3] == again[3]


def test_phased_subjects_match_oracle(mpm):
    gn, cg = 4, 30
    # one group of two (K = 4, 16 x 16 tiles), both with a variance output
    subs = [_subject(mpm, s)[:3] + (True,) for s in (SUBJECTS[3], SUBJECTS[6])]
    ys, vs, reps, _ = _batch(mpm, subs, mpm.make_opts(gn_iters=gn, cg_iters=cg, graph="phased"))
    for (d, pg, _, with_var), y, var, rep in zip(subs, ys, vs, reps):
        po = orc.make_problem(d["prot"], d["shape"])
        ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=gn, cg_iters=cg)
        np.testing.assert_allclose(np.array(rep.F[:gn + 1]), ref["F"], rtol=1e-5)
        assert map_error(to_np(y), ref["y"]).max() <= 1e-3
        # the posterior variance (Eq. 43) at the oracle's final maps
        _, _, h = orc.grad_hess(po, d["x"], ref["y"], d["b1p"], d["b1m"])
        _, w = orc.jtv(po, ref["y"])
        var_o, _, _, _ = orc.uncertainty(po, h, w)
        np.testing.assert_allclose(to_np(var), var_o, rtol=5e-3)


def test_groups_of_sixteen(mpm):
    """Eighteen small subjects of one class: a group of 16 and one of 2."""
    gn, cg = 3, 12
    specs = [((24 + 4 * (i % 3), 18 + i, 6 + i % 4), 200 + i, ("PDw", "T1w", "MTw"), (4, 4, 3),
              False, i % 2 == 0) for i in range(18)]
    subs = [_subject(mpm, s) for s in specs]
    solos = [_solo(mpm, d, pg, x, v, mpm.make_opts(gn_iters=gn, cg_iters=cg)) for d, pg, x, v in subs]
    ys, vs, reps, launches = _batch(mpm, subs, mpm.make_opts(gn_iters=gn, cg_iters=cg, graph="phased"))
    for i, (sol, yb, vb, rb) in enumerate(zip(solos, ys, vs, reps)):
        _check_equal_to_solo(sol, yb, vb, rb, gn, i)
    assert launches == 2 * _launches_per_group(gn, cg, True) + INIT_LAUNCHES * 18, launches


def test_unaligned_subject_runs_in_a_lane(mpm):
    """A volume whose x size is not a multiple of 4 cannot use the staged
    iteration: it runs in a lane of its own (as with graph = 1, its solo
    result bit for bit) beside the group of the two others."""
    spec = ((33, 17, 9), 92, ("PDw", "T1w"), (6, 4), False, True)
    subs = [_subject(mpm, spec), _subject(mpm, SUBJECTS[0]), _subject(mpm, SUBJECTS[4])]
    gn, cg = 3, 15
    solos = [_solo(mpm, d, pg, x, v, mpm.make_opts(gn_iters=gn, cg_iters=cg)) for d, pg, x, v in subs]
    ys, vs, reps, launches = _batch(mpm, subs, mpm.make_opts(gn_iters=gn, cg_iters=cg, graph="phased"))
    y, var, rep = solos[0]
    assert np.array_equal(to_np(y), to_np(ys[0]))
    assert np.array_equal(to_np(var), to_np(vs[0]))
    assert list(rep.F[:gn + 1]) == list(reps[0].F[:gn + 1])
    for i in (1, 2):
        _check_equal_to_solo(solos[i], ys[i], vs[i], reps[i], gn, i)
    assert launches == 2 * _launches_per_group(gn, cg, True) + INIT_LAUNCHES * 3, launches


def test_single_fit_with_the_phased_graph(mpm):
    """mpm_fit with opts.graph = 2: a group of one subject, which the wave
    split gives the solo grid; the result meets the fit tolerances of the
    direct-launch fit."""
    gn, cg = 4, 30
    d, pg, x, v = _subject(mpm, SUBJECTS[0])
    solo = _solo(mpm, d, pg, x, v, mpm.make_opts(gn_iters=gn, cg_iters=cg))
    y, var, rep = _solo(mpm, d, pg, x, v, mpm.make_opts(gn_iters=gn, cg_iters=cg, graph="phased"))
    _check_equal_to_solo(solo, y, var, rep, gn, "phased single")
