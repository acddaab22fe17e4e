"""me_acbm_noalloc: the ACBM entry point for callers that cannot allocate
device memory (engines or plugins that own every allocation under a fixed
budget, code that must not allocate after start-up).  It keeps its scratch in
a fixed 4 MiB device array inside the library.

Checked through the C ABI against me_acbm (the allocating entry point) on two
calls in a row, bit for bit, as every other parity test here.  The file is
named to be collected last, and it passes alone in a fresh process as well
as after the other tests (the first call does the per-device set-up).
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _run(lib, fn, cur, ref, N, M, p, lam, prm, prev):
    import torch
    H, W = cur.shape
    BH, BW = H // M, W // N
    mv = torch.full((BH, BW, 2), -999, dtype=torch.int16, device="cuda")
    J = torch.full((BH, BW), -1, dtype=torch.int32, device="cuda")
    mask = torch.full((BH, BW), 7, dtype=torch.uint8, device="cuda")
    sad = torch.full((BH, BW), -1, dtype=torch.int32, device="cuda")
    load = torch.full((BH, BW), -1, dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    st = getattr(lib, fn)(vp(cur.data_ptr()), vp(ref.data_ptr()), W, H, N, M, p, lam,
                          None if prev is None else vp(prev.data_ptr()), ctypes.byref(prm),
                          vp(mv.data_ptr()), vp(J.data_ptr()), vp(mask.data_ptr()),
                          vp(sad.data_ptr()), vp(load.data_ptr()),
                          vp(torch.cuda.current_stream().cuda_stream))
    assert st == 0, (fn, st)
    torch.cuda.synchronize()
    return mv, [t.cpu().numpy() for t in (mv, J, mask, sad, load)]


@pytest.mark.parametrize("name,p,qp,N,M", [("cif", 16, 28, 16, 16), ("1080p", 32, 28, 16, 16),
                                           ("1080p", 64, 28, 8, 8)])
def test_noalloc_matches_acbm_on_consecutive_calls(name, p, qp, N, M):
    import torch
    import paper_0710_4819_gb300 as me
    lib = me.load_library(build_if_missing=True)
    seq = synth.config_sequence(name, seed=31, n_frames=3)
    frames = torch.from_numpy(seq).cuda()
    lam = me.me_lambda_q8(qp)
    prm = me.params(qp=qp)
    prev_a = prev_n = None
    for t in (1, 2):          # two calls in a row, the second chained on the first
        mv_a, want = _run(lib, "me_acbm", frames[t], frames[t - 1], N, M, p, lam, prm, prev_a)
        mv_n, got = _run(lib, "me_acbm_noalloc", frames[t], frames[t - 1], N, M, p, lam, prm,
                         prev_n)
        for nm, g, w in zip(("mv", "J", "mask", "sad", "load"), got, want):
            assert np.array_equal(g, w), f"{name} t={t}: {nm} differs"
        prev_a, prev_n = mv_a, mv_n


@pytest.mark.parametrize("W,H,N,M,p", [(3840, 2160, 16, 16, 64), (1920, 1088, 4, 4, 16)])
def test_noalloc_rejects_frames_beyond_its_array(W, H, N, M, p):
    """2160p at 16x16 and 1080p at 4x4 blocks need more than the 4 MiB array
    (9.3 and 4.6 MB): refused with ME_ERR_NOMEM, nothing enqueued."""
    import torch
    import paper_0710_4819_gb300 as me
    lib = me.load_library(build_if_missing=True)
    x = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    out = torch.zeros((H // M, W // N, 2), dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    prm = me.params(qp=28)
    st = lib.me_acbm_noalloc(vp(x.data_ptr()), vp(x.data_ptr()), W, H, N, M, p, 6595,
                             None, ctypes.byref(prm), vp(out.data_ptr()), vp(out.data_ptr()),
                             vp(out.data_ptr()), None, None,
                             vp(torch.cuda.current_stream().cuda_stream))
    assert st == 4   # ME_ERR_NOMEM: the frame needs more scratch than the fixed array holds
