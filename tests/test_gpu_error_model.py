"""The float32 error model behind the oracle's ambiguity flags, checked on the
GPU's own quantities.  A decision (cull, tile edge, alpha skip, transmittance
stop, depth order) is flagged only when it lies closer to its threshold than
these bounds, so every bound the oracle assumes is tested here against what
the kernels actually compute:

- camera depth keys: the correctly rounded float of the FP64 camera depth
  (the compensated transform), so the per-tile depth order is the oracle's;
- image position u, v: within ratio u fx |p_x / p_z| + round u |u|;
- conic: as a quadratic form within conic u sqrt(kappa) (relative), kappa
  the condition number of the 2D covariance;
- opacity: within opacity u (relative);
- the exponential of alpha = o exp(-sigma): within exp (relative) for sigma
  in [0, 6], the range in which a skip or stop decision can be marginal
  (alpha >= 1/255 needs sigma <= ln 255 < 5.55).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2312_10070_gb300 import _lib, api, synth as S
from tests.gpu_common import ocam, unit_inputs

pytestmark = pytest.mark.gpu


def test_exponential_within_the_assumed_bound():
    em = O.error_model()
    lib = _lib.load()
    sig = np.concatenate([np.linspace(0.0, 6.0, 2_000_001), np.random.default_rng(0).uniform(0, 6, 4_000_000)])
    x = (-sig).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    st = lib.gsr_probe_expf(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.size,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    ref = np.exp(x.astype(np.float64))
    rel = np.abs(y.cpu().numpy().astype(np.float64) - ref) / ref
    print("exponential: max relative error", rel.max(), "bound", em["exp"])
    assert rel.max() <= em["exp"]


def _records_vs_model(sc, spec, q, t, tile):
    em = O.error_model()
    U = em["u"]
    ctx = api.Context(tile=tile)
    g = api.GaussianParams.from_numpy(sc)
    api.render_forward(ctx, g, api.camera_from_spec(spec), api.make_pose(q, t))
    torch.cuda.synchronize()
    rec, vis = api.records(ctx, g.n)
    ctx.close()
    sc64 = O.Scene.from_dict(sc)
    pr = O.project(sc64, q, t, ocam(spec, tile))
    unsure = (pr["amb"] & 1).astype(bool)
    assert np.array_equal(vis[~unsure], pr["visible"][~unsure].astype(bool))
    m = vis & (pr["visible"] == 1)
    # depth keys: correctly rounded
    key = rec[m, 6].view(np.uint32)
    assert np.array_equal(key, pr["depth"][m].astype(np.float32).view(np.uint32))
    # u, v
    uv = pr["uv"][m]
    for k, f, c in ((0, spec.fx, spec.cx), (1, spec.fy, spec.cy)):
        ratio = (uv[:, k] - c) / f
        bound = em["ratio"] * U * f * np.abs(ratio) + em["round"] * U * np.abs(uv[:, k]) + 1e-9
        err = np.abs(rec[m, k].astype(np.float64) - uv[:, k])
        print("uv", k, "max error / bound", (err / bound).max())
        assert (err <= bound).all()
    # conic as a quadratic form: eigenvalues of C^-1/2 (C_gpu - C) C^-1/2
    A, B, C = pr["conic"][m].T
    a, b, c = (rec[m, k].astype(np.float64) for k in (2, 3, 4))
    M = np.stack([np.stack([A, B], -1), np.stack([B, C], -1)], -2)
    D = np.stack([np.stack([a - A, b - B], -1), np.stack([b - B, c - C], -1)], -2)
    Li = np.linalg.inv(np.linalg.cholesky(M))
    rho = np.abs(np.linalg.eigvalsh(Li @ D @ np.swapaxes(Li, -1, -2))).max(-1)
    ev = np.linalg.eigvalsh(M)
    bound = em["conic"] * U * np.sqrt(ev[:, 1] / ev[:, 0])
    print("conic max error / bound", (rho / bound).max())
    assert (rho <= bound).all()
    # opacity
    eo = np.abs(rec[m, 5].astype(np.float64) - pr["opacity"][m]) / pr["opacity"][m]
    print("opacity max error / bound", eo.max() / (em["opacity"] * U))
    assert (eo <= em["opacity"] * U).all()


@pytest.mark.parametrize("seed,pose_seed", [(1, 2), (7, 8), (3, 4)])
def test_unit_scene_records_within_the_error_model(seed, pose_seed):
    sc, spec, q, t = unit_inputs(seed, pose_seed)
    _records_vs_model(sc, spec, q, t, (16, 16))


def test_room_view_records_within_the_error_model():
    q, t = S.submap_views()[S.HEADLINE_VIEW]
    _records_vs_model(S.room_scene(500_000, seed=3), S.camera_room(), q, t, (8, 8))
