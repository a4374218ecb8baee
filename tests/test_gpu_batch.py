"""Batched fits and CUDA-graph replay.

Several subjects of different sizes, contrasts, echo counts and echo storage
are fitted in one mpm_fit_batch call (their updates captured as parallel
branches of one CUDA graph).  Every subject must give exactly its solo
mpm_fit result, which in turn matches the FP64 oracle; a graph replay (cache
hit) must repeat the first run bit for bit.
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


SUBJECTS = [
    # shape, seed, contrasts, echoes, bf16 echoes
    ((48, 40, 20), 91, ("PDw", "T1w", "MTw"), (8, 8, 6), False),
    ((33, 17, 9), 92, ("PDw", "T1w"), (6, 4), False),
    ((64, 24, 12), 93, ("PDw", "T1w", "MTw"), (5, 7, 4), True),
    ((20, 20, 20), 94, ("PDw", "T1w", "MTw", "VFA15"), (4, 4, 4, 4), False),
]


def _subject(mpm, spec):
    import torch
    shape, seed, contrasts, echoes, bf16 = spec
    d = dataset(shape, seed=seed, contrasts=contrasts, n_echoes=echoes)
    pg = mpm.make_problem(d["prot"], shape, echo_dtype=1 if bf16 else 0)
    x = to_dev(d["x"])
    if bf16:
        x = x.to(torch.bfloat16)
        d["x"] = x.float().cpu().numpy()
    return d, pg, x


def _solo(mpm, d, pg, x, opts):
    import torch
    N = int(np.prod(d["shape"]))
    y = torch.zeros((pg.n_maps, N), dtype=torch.float32, device="cuda")
    var = torch.zeros((pg.n_maps, N), dtype=torch.float32, device="cuda")
    st, rep = mpm.mpm_fit(pg, opts, x, y, to_dev(d["b1p"]), to_dev(d["b1m"]), var=var)
    return y, var, rep


def test_graph_replay_matches_direct_launches(mpm):
    d, pg, x = _subject(mpm, SUBJECTS[0])
    y0, v0, r0 = _solo(mpm, d, pg, x, mpm.make_opts(gn_iters=5, cg_iters=30))
    for _ in range(2):                      # capture, then replay from the cache
        y1, v1, r1 = _solo(mpm, d, pg, x, mpm.make_opts(gn_iters=5, cg_iters=30, graph=True))
        assert np.array_equal(to_np(y0), to_np(y1))
        assert np.array_equal(to_np(v0), to_np(v1))
        assert list(r0.F[:6]) == list(r1.F[:6])


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_solo_fits(mpm, graph):
    import torch
    opts = mpm.make_opts(gn_iters=6, cg_iters=30, graph=graph)
    subs = [_subject(mpm, s) for s in SUBJECTS]
    solos = [_solo(mpm, d, pg, x, mpm.make_opts(gn_iters=6, cg_iters=30)) for d, pg, x in subs]
    ys = [torch.zeros_like(s[0]) for s in solos]
    vs = [torch.zeros_like(s[1]) for s in solos]
    st, reps = mpm.mpm_fit_batch([pg for _, pg, _ in subs], opts, [x for _, _, x in subs], ys,
                                 b1ps=[to_dev(d["b1p"]) for d, _, _ in subs],
                                 b1ms=[to_dev(d["b1m"]) for d, _, _ in subs], vars=vs)
    for i, ((y, v, rep), yb, vb, rb) in enumerate(zip(solos, ys, vs, reps)):
        assert rb.iters == rep.iters == 6
        assert np.array_equal(to_np(y), to_np(yb)), i
        assert np.array_equal(to_np(v), to_np(vb)), i
        assert list(rep.F[:7]) == list(rb.F[:7]), i


def test_batch_subjects_match_oracle(mpm):
    import torch
    subs = [_subject(mpm, s) for s in SUBJECTS[1:3]]
    opts = mpm.make_opts(gn_iters=4, cg_iters=30, graph=True)
    ys = [torch.zeros((pg.n_maps, int(np.prod(d["shape"]))), device="cuda") for d, pg, _ in subs]
    st, reps = mpm.mpm_fit_batch([pg for _, pg, _ in subs], opts, [x for _, _, x in subs], ys,
                                 b1ps=[to_dev(d["b1p"]) for d, _, _ in subs],
                                 b1ms=[to_dev(d["b1m"]) for d, _, _ in subs])
    for (d, pg, _), y, rep in zip(subs, ys, reps):
        po = orc.make_problem(d["prot"], d["shape"])
        ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=4, cg_iters=30)
        np.testing.assert_allclose(np.array(rep.F[:5]), ref["F"], rtol=1e-5)
        assert map_error(to_np(y), ref["y"]).max() <= 1e-3
