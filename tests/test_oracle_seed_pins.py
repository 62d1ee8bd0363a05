"""Pins of the FP64 seeding oracle (oracle/seed.py), CPU only: the
generator's published outputs and bijectivity, sampling-set properties, the
gradient on a linear ramp, back-projection round trips through the pinhole,
and nearest-neighbour / radius decisions against scipy's k-d tree."""
import json
import os
from types import SimpleNamespace

import numpy as np
from scipy.spatial import cKDTree

from oracle import seed as SD

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = 0x9E3779B97F4A7C15


def test_splitmix64_published_outputs_and_bijectivity():
    gold = json.load(open(os.path.join(HERE, "golden", "splitmix64.json")))
    got = [int(SD.splitmix64(np.uint64((k * GOLD) % (1 << 64)))) for k in range(3)]
    assert got == [int(h, 16) for h in gold["outputs_hex"]]
    x = SD.splitmix64(np.arange(1 << 20, dtype=np.uint64))
    assert np.unique(x).size == 1 << 20                      # a bijection: no collisions
    bits = ((x[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.005)                # every output bit balanced


def test_sampling_keys_are_the_published_generator_outputs():
    """The key of pixel 0 under seed k * gamma is the k-th published output of
    SplitMix64 seeded with 0, high 32 bits."""
    gold = json.load(open(os.path.join(HERE, "golden", "splitmix64.json")))
    for k, h in enumerate(gold["outputs_hex"]):
        assert int(SD.uniform_keys(1, (k * GOLD) % (1 << 64))[0]) == int(h, 16) >> 32


def test_uniform_sample_is_an_exact_nested_uniform_subset():
    rng = np.random.default_rng(0)
    elig = rng.random(4000) < 0.6
    a = SD.sample_uniform(elig, 500, seed=7)
    b = SD.sample_uniform(elig, 900, seed=7)
    # the sample is the m eligible pixels of smallest key: no unselected
    # eligible pixel has a smaller key than a selected one
    keys = SD.uniform_keys(4000, 7).astype(np.int64)
    rest = np.setdiff1d(np.nonzero(elig)[0], a)
    assert keys[a].max() <= keys[rest].min()
    assert a.size == 500 and b.size == 900 and np.all(elig[a])
    assert np.all(np.diff(a) > 0) and set(a) <= set(b)       # ascending, nested
    np.testing.assert_array_equal(SD.sample_uniform(elig, 10 ** 6, 3), np.nonzero(elig)[0])
    # every eligible pixel is picked with probability m / n over seeds
    cnt = np.zeros(4000)
    for s in range(400):
        cnt[SD.sample_uniform(elig, 600, seed=1000 * s)] += 1
    n = elig.sum()
    p = 600 / n
    z = (cnt[elig] - 400 * p) / np.sqrt(400 * p * (1 - p))
    assert abs(z.mean()) < 0.1 and 0.8 < z.std() < 1.2
    assert cnt[~elig].sum() == 0


def test_gradient_of_a_linear_ramp_and_top_m_selection():
    H, W = 9, 12
    i, j = np.mgrid[0:H, 0:W]
    y = 0.03 * j - 0.02 * i + 0.5
    rgb = np.stack([y, y, y])
    g = SD.gradient2(rgb)
    np.testing.assert_allclose(g[1:-1, 1:-1], 0.03 ** 2 + 0.02 ** 2, rtol=1e-12)
    assert np.all(g[0] == 0) and np.all(g[-1] == 0) and np.all(g[:, 0] == 0) and np.all(g[:, -1] == 0)
    g2 = np.zeros((H, W))
    g2[2, 3], g2[5, 7], g2[6, 1] = 3.0, 2.0, 2.0
    top = SD.sample_gradient(np.ones((H, W), bool), g2, 2)
    np.testing.assert_array_equal(top, [2 * W + 3, 5 * W + 7])   # tie 2.0: the smaller pixel index wins
    top = SD.sample_gradient(np.ones((H, W), bool), g2, 3)
    np.testing.assert_array_equal(top, sorted([2 * W + 3, 5 * W + 7, 6 * W + 1]))


def _quat(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * a])


def test_backprojection_round_trips_through_the_pinhole():
    cam = SimpleNamespace(fx=150.0, fy=140.0, cx=80.0, cy=60.0)
    rng = np.random.default_rng(1)
    depth = rng.uniform(0.5, 5.0, (120, 160))
    q, t = _quat([0.3, -1, 0.2], 0.7), np.array([0.4, -0.2, 1.1])
    pix = rng.choice(120 * 160, 300, replace=False)
    pw = SD.backproject(pix, depth, cam, q, t)
    R = SD._rot(q)
    pc = pw @ R.T + t
    i, j = np.divmod(pix, 160)
    np.testing.assert_allclose(pc[:, 2], depth.ravel()[pix], rtol=1e-12)
    np.testing.assert_allclose(cam.fx * pc[:, 0] / pc[:, 2] + cam.cx, j + 0.5, atol=1e-9)
    np.testing.assert_allclose(cam.fy * pc[:, 1] / pc[:, 2] + cam.cy, i + 0.5, atol=1e-9)


def test_distances_and_keyframe_seeding_against_kdtree():
    rng = np.random.default_rng(2)
    H, W = 40, 60
    cam = SimpleNamespace(fx=50.0, fy=50.0, cx=30.0, cy=20.0)
    depth = rng.uniform(1.0, 1.2, (H, W))
    depth[rng.random((H, W)) < 0.1] = 0.0
    rgb = rng.random((3, H, W))
    q, t = _quat([0, 0, 1], 0.0), np.zeros(3)
    existing = rng.uniform([-0.6, -0.4, 0.9], [0.6, 0.4, 1.3], (3000, 3))
    out = SD.seed_keyframe(rgb, depth, None, cam, q, t, existing, first=True, m_u=600, m_c=200, rho=0.03,
                           s_max=0.2, seed=5)
    pts = out["points"]
    assert np.all(depth.ravel()[out["pix"]] > 0)
    tree = cKDTree(existing)
    d, _ = tree.query(pts)
    np.testing.assert_allclose(np.sqrt(out["d2_existing"]), d, rtol=1e-12)
    np.testing.assert_array_equal(out["keep"], d >= 0.03)
    new = pts[out["keep"]]
    union = np.concatenate([existing, new])
    dn, _ = cKDTree(union).query(new, k=2)   # the first hit is the point itself
    s = np.clip(dn[:, 1], 1e-4, 0.2)
    np.testing.assert_allclose(out["gaussians"]["log_scale"], np.log(s)[:, None].repeat(3, 1), rtol=1e-12)
    np.testing.assert_array_equal(out["gaussians"]["rgb"], rgb.reshape(3, -1)[:, out["pix"][out["keep"]]].T)
    # later keyframe: only pixels whose alpha is below alpha_n
    alpha = rng.random((H, W))
    out2 = SD.seed_keyframe(rgb, depth, alpha, cam, q, t, existing, first=False, m_k=300, rho=0.03, seed=6)
    assert out2["pix"].size == 300 and np.all(alpha.ravel()[out2["pix"]] < 0.6)


def test_merge_rule_on_a_constructed_case():
    rho = 0.01
    a = dict(mean=np.array([[0.0, 0, 0], [1.0, 0, 0]]), rgb=np.array([[1.0, 0, 0], [0, 1.0, 0]]))
    b = dict(mean=np.array([[0.005, 0, 0],      # within rho of a[0]: dropped
                            [0.0, 0.0101, 0],   # just outside rho of a[0]: kept
                            [2.0, 0, 0], [2.001, 0, 0]]),  # near each other only: both kept
             rgb=np.zeros((4, 3)))
    merged, masks = SD.merge([a, b], rho)
    np.testing.assert_array_equal(masks[0], [True, True])
    np.testing.assert_array_equal(masks[1], [False, True, True, True])
    assert merged["mean"].shape == (5, 3)
    # against scipy's k-d tree on random data
    rng = np.random.default_rng(3)
    s1 = dict(mean=rng.uniform(0, 0.3, (2000, 3)))
    s2 = dict(mean=rng.uniform(0.1, 0.4, (2000, 3)))
    _, m = SD.merge([s1, s2], 0.01)
    d, _ = cKDTree(s1["mean"]).query(s2["mean"])
    np.testing.assert_array_equal(m[1], d >= 0.01)


def test_prune_keeps_exactly_the_logits_above_the_threshold_in_order():
    """Opacity sigmoid(logit) >= o_min  <=>  logit >= ln(o_min / (1 - o_min)):
    the kept set is fixed by the closed-form inverse, order and pairing kept."""
    rng = np.random.default_rng(4)
    n = 5000
    params = dict(mean=rng.standard_normal((n, 3)), log_scale=rng.standard_normal((n, 3)),
                  quat=rng.standard_normal((n, 4)), opacity_logit=rng.normal(0.0, 3.0, n),
                  rgb=rng.random((n, 3)))
    for o_min in (0.1, 0.005, 0.6):
        thr = np.log(o_min / (1 - o_min))
        far = np.abs(params["opacity_logit"] - thr) > 1e-9
        out, keep = SD.prune(params, o_min)
        np.testing.assert_array_equal(keep[far], params["opacity_logit"][far] >= thr)
        for k, v in params.items():
            np.testing.assert_array_equal(out[k], v[keep])   # same rows, original order
