"""The Table 1 layout (ACBM candidate positions per block against Qp, at 30
and 10 fps) on the synthetic QCIF load scenes: every cell's per-block
outputs from the one-launch sequence form equal the oracle chained pair by
pair, and the table shows the trends Sec. 4 reports (load falls as Qp
rises, rises at the lower frame rate, and is lowest for the smooth slow
scene and highest for the textured fast one)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

P = 15


@pytest.fixture(scope="module")
def me():
    import torch
    assert torch.cuda.is_available()
    import paper_0710_4819_gb300 as me
    me.load_library(build_if_missing=True)
    return me


def _gpu(me, frames, qp):
    import torch
    a = me.me_acbm_sequence(torch.from_numpy(frames).cuda(), 16, 16, P, me.me_lambda_q8(qp),
                            me.params(qp=qp))
    torch.cuda.synchronize()
    return (a.mv.cpu().numpy(), a.J.cpu().numpy().view(np.uint32), a.mask.cpu().numpy(),
            a.sad.cpu().numpy().view(np.uint32), a.load.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("name", sorted(synth.LOAD_RECIPES))
@pytest.mark.parametrize("fps", [30, 10])
def test_load_cells_match_chained_oracle(me, orc, name, fps):
    frames = synth.load_sequence(name, fps, seed=500)
    for qp in (30, 22, 16):
        got = _gpu(me, frames, qp)
        prev = None
        lam = orc.lambda_q8(qp)
        for k in range(1, len(frames)):
            want = orc.acbm(frames[k], frames[k - 1], 16, 16, P, lam, orc.params(qp=qp), prev)
            prev = want[0]
            for i, tag in enumerate(("mv", "J", "mask", "sad", "load")):
                assert np.array_equal(got[i][k - 1], want[i]), (name, fps, qp, k, tag)


def test_load_table_trends(me):
    qps = (30, 26, 22, 16)
    tab = {}
    for name in synth.LOAD_RECIPES:
        for fps in (30, 10):
            frames = synth.load_sequence(name, fps, seed=500)
            tab[name, fps] = [float(_gpu(me, frames, qp)[4].mean()) for qp in qps]
    for key, row in tab.items():
        assert all(a <= b for a, b in zip(row, row[1:])), (key, row)     # Qp falls -> load rises
        assert row[0] < row[-1], (key, row)
    for name in synth.LOAD_RECIPES:
        assert sum(tab[name, 10]) > sum(tab[name, 30]), name
    tot = {name: sum(tab[name, 30]) + sum(tab[name, 10]) for name in synth.LOAD_RECIPES}
    assert min(tot, key=tot.get) == "smooth-slow" and max(tot, key=tot.get) == "textured-fast"
    # every cell far below the full search's (2p+1)^2 = 961
    assert max(max(r) for r in tab.values()) < 961 / 2
