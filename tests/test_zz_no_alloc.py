"""kf_reduce_noalloc: the reduction for callers that cannot allocate device memory.

Some callers run inside a host application whose CUDA allocator belongs to
another runtime, or may not add cudaMalloc / cudaFree synchronisation while
their other work is in flight; this entry point works on their buffers only and
keeps its scratch in a fixed array inside the library. The test feeds it the
maps a tracker built, with model holes that the caller made (a finite vertex
beside a NaN normal, and an all-zero normal), and checks its sums against the
oracle's sums on the same maps, within the tolerance the other reduction tests
use. Calls are queued back to back on one stream: two at full size, then two
on a smaller level, so the small calls run right after a larger one left its
partial sums in the shared array. The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from oracle import kf_oracle as O
from synth import scenes as S
from tests import kfhelp as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03980_gb300 import build
    build()


def test_noalloc_reduction_matches_the_oracle_on_calls_in_a_row():
    import torch
    k = H.kf()
    pr = S.config2_kinect(3, 640, 480)
    p, op = H.params()
    with H.Tracker(p, 640, 480) as t:
        t.set_pair(pr)
        fr, mo = H.oracle_levels_from_gpu(t, pr, 3)
    T = O.seed_pose(pr.prior_R, pr.init_pose, op)
    cases = []
    for l in (0, 2):
        mc = mo[l].cam
        a0 = O.associate(fr[l], mo[l], T, O.f32_transforms(T, pr.model_pose), op)
        # holes the caller made at matched model pixels
        V = np.array(mo[l].V, np.float64)
        N = np.array(mo[l].N, np.float64)
        hit = np.unique(a0.vi[a0.valid] * mc.width + a0.ui[a0.valid])
        nan_n, zero_n = hit[::97], hit[5::89]
        N.reshape(-1, 3)[nan_n, 1] = np.nan
        N.reshape(-1, 3)[zero_n] = 0.0
        assert np.isfinite(V.reshape(-1, 3)[nan_n]).all()
        ml = O.ModelLevel(V, N, mc)
        a = O.associate(fr[l], ml, T, O.f32_transforms(T, pr.model_pose), op)
        assert a.valid.sum() < a0.valid.sum()
        kmed = O.median_bin(O.histogram(a, p.hist_bins))
        klo, khi = O.band(kmed, 1.0, p.hist_bins)
        want, A, bb = H.oracle_sums(a, a.valid & (a.k >= klo) & (a.k <= khi))
        tol = H.sum_tolerances(A, bb)
        h, w = fr[l].V.shape[:2]
        cases.append(dict(
            l=l, w=w, h=h, mc=mc, klo=klo, khi=khi, want=want, tol=tol,
            fv=torch.from_numpy(np.ascontiguousarray(fr[l].V, np.float32)).cuda(),
            mv=torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda(),
            mn=torch.from_numpy(np.ascontiguousarray(N, np.float32)).cuda()))
    out = torch.full((4, 29), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    row = 0
    for c in cases:  # level 0 (75 blocks) twice, then level 2 (5 blocks) twice
        mc = c["mc"]
        for _ in range(2):
            st = k.kf_reduce_noalloc(c["fv"].data_ptr(), c["w"], c["h"], c["mv"].data_ptr(),
                                     c["mn"].data_ptr(),
                                     (mc.width, mc.height, mc.fx, mc.fy, mc.cx, mc.cy), T,
                                     pr.model_pose, p.d_max, p.hist_bins, c["klo"], c["khi"],
                                     out[row].data_ptr(), 0)
            assert st == k.KF_OK
            row += 1
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i, c in enumerate(cases):
        for call in range(2):
            g = got[2 * i + call]
            assert np.isfinite(g).all(), (c["l"], call)
            assert g[27] == c["want"][27], (c["l"], call)
            assert (np.abs(g - c["want"]) <= c["tol"]).all(), (c["l"], call)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    k = H.kf()
    st = k.kf_reduce_noalloc(1, 4096, 1025, 1, 1, (64, 48, 50.0, 50.0, 32.0, 24.0), np.eye(4),
                             np.eye(4), 0.16, 512, 0, 10, 1, 0)
    assert st == k.KF_ERR_SCRATCH_LIMIT
