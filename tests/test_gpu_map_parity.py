"""The mapping step as the benchmark times it, against the oracle's chain.

gsr_map_step with one keyframe runs the fused projection backward + Adam
kernel (the gradients never leave registers); with several it runs the
persistent (keyframe, tile) blends and the separate Adam.  Both are compared
with the FP64 oracle's plain chain of Sec. 3.2 / 3.4 (Eq. (joint_loss) and
L_reg): render -> mapping loss (L1 colour, SSIM, L1 depth over valid pixels)
-> render backward, summed over keyframes with their weights, + the L_reg
gradient -> bias-corrected Adam with the per-group learning rates.

Compared element by element after the step: the loss, the Adam moments (the
first moment is (1 - beta1) g, so it carries the gradient; the second
(1 - beta2) g^2) and every parameter.  At the first step Adam moves a
parameter by lr sign(g), so a parameter must match the oracle's exactly
(up to float rounding) wherever the gradient bar fixes the sign of g; where
it does not (|g| within the bar of 0) the step must still have size lr, and
where g = 0 the parameter must not move.

Targets are the oracle's renders from another pose, pushed at least 0.01 away
from the render being optimised wherever they are closer, so the sign of
every L1 residual is fixed by the 2e-4 image bar.  At pixels where a skip or
stop decision is marginal, the oracle takes the branches the GPU's forward
took (check_forward); the map step's forward runs the same kernels as
gsr_render_forward, whose output gives those branches.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2312_10070_gb300 import api, synth as S
from tests.gpu_common import check_forward, grad_close, ocam, strict_pass_fraction, unit_inputs

pytestmark = pytest.mark.gpu

GROUPS = (("mean", "lr_mean"), ("log_scale", "lr_log_scale"), ("quat", "lr_quat"), ("opacity_logit", "lr_opacity"),
          ("rgb", "lr_rgb"))


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def margin_target(r_rgb, r_d, t_rgb, t_d, margin=0.01):
    """A target whose L1 residuals against the render (r_rgb, r_d) are at
    least `margin` in magnitude (colour everywhere, depth where the target
    depth is valid), float32."""
    s = np.where(r_rgb < 0.5, 1.0, -1.0)
    rgb = np.where(np.abs(r_rgb - t_rgb) < margin, r_rgb + s * margin, t_rgb)
    d = np.where((t_d > 0) & (np.abs(r_d - t_d) < margin), r_d + margin, t_d)
    return rgb.astype(np.float32), d.astype(np.float32)


def gpu_flips(ctx, g, cam, q, t, sc64, oc, label, max_excluded=0.0):
    out = api.render_forward(ctx, g, cam, api.make_pose(q, t), want_n_contrib=True)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    flips, excl, ref = check_forward(ctx, out, sc64, q, t, oc, max_excluded=max_excluded, label=label)
    return flips, excl, ref


def oracle_grads(sc64, views, oc, weights, cfg):
    """Weighted mapping loss + w_reg L_reg and its gradient (oracle chain);
    views = [(q, t, rgb_target, depth_target, flips)]."""
    total = {k: np.zeros_like(getattr(sc64, k)) for k, _ in GROUPS}
    L = 0.0
    for (q, t, rgb_t, d_t, fl), w in zip(views, weights):
        r = O.render(sc64, q, t, oc, flips=fl)
        lm = O.loss_map(r["rgb"], r["depth"], rgb_t, d_t, cfg.lambda_ssim, cfg.w_color, cfg.w_depth)
        gb = O.render_backward(sc64, q, t, oc, w * lm["d_rgb"], w * lm["d_depth"], None, flips=fl)
        L += w * lm["loss"]
        for k in total:
            total[k] += gb[k].reshape(total[k].shape)
    Lr, greg = O.lreg(sc64.log_scale, cfg.adam.w_reg)
    total["log_scale"] += greg
    return L + cfg.adam.w_reg * Lr, total


def oracle_adam(params, grads, m, v, step, cfg):
    a = cfg.adam
    for k, lrk in GROUPS:
        O.adam(params[k], np.ascontiguousarray(grads[k]), m[k], v[k], step, getattr(a, lrk), a.beta1, a.beta2, a.eps)


def restore(g, st, init):
    for dst, src in zip(g.tensors(), init.tensors()):
        dst.copy_(src)
    for tt in st.m.tensors() + st.v.tensors():
        tt.zero_()
    st.step.zero_()


def check_first_step(g, st, sc0, grads, cfg, label):
    """Moments and parameters after one Adam step against the oracle's."""
    a = cfg.adam
    for k, lrk in GROUPS:
        lr = getattr(a, lrk)
        gr = grads[k].reshape(-1)
        m = getattr(st.m, k).cpu().numpy().reshape(-1).astype(np.float64)
        v = getattr(st.v, k).cpu().numpy().reshape(-1).astype(np.float64)
        ok, worst = grad_close(m / (1 - a.beta1), gr)
        strict = strict_pass_fraction(m / (1 - a.beta1), gr)
        print(f"{label} {k}: gradient (first moment) worst ratio {worst:.3f}, strict-floor pass {strict:.5f}")
        assert ok, (label, k, "first moment", worst)
        assert strict >= 0.995, (label, k, "strict floor", strict)
        ok, worst = grad_close(np.sqrt(v / (1 - a.beta2)), np.abs(gr))
        assert ok, (label, k, "second moment", worst)
        th0 = getattr(sc0, k).reshape(-1)
        th_ref = th0 - lr * gr / (np.abs(gr) + a.eps)
        th = getattr(g, k).detach().cpu().numpy().reshape(-1).astype(np.float64)
        tol_g = 1e-3 * (np.abs(gr) + 0.1 * np.abs(gr).max())
        det = np.abs(gr) > tol_g
        ulp = np.spacing(np.abs(th_ref).astype(np.float32)).astype(np.float64)
        err = np.abs(th - th_ref)
        assert (err[det] <= 2e-6 * lr + ulp[det]).all(), (label, k, "determined", err[det].max() / lr)
        zero = gr == 0
        assert (th[zero] == th0[zero]).all(), (label, k, "zero gradient moved")
        rest = ~det & ~zero
        assert (np.abs(th[rest] - th0[rest]) <= lr * (1 + 1e-5) + ulp[rest]).all(), (label, k, "step size")
        print(f"{label} {k}: {det.sum()} parameters with a determined step match, {rest.sum()} undetermined, "
              f"{zero.sum()} untouched")


def unit_map_inputs(seed=1, pose_seed=2):
    """Unit scene rendered at a perturbed pose against a target rendered
    from the identity pose (the single-frame workload's recipe)."""
    sc, spec, q, t = unit_inputs(seed, pose_seed)
    sc64 = O.Scene.from_dict(sc)
    oc = ocam(spec)
    r = O.render(sc64, q, t, oc)
    tg = O.render(sc64, *S.IDENTITY_POSE, oc)
    rgb_t, d_t = margin_target(r["rgb"], r["depth"], tg["rgb"], tg["depth"])
    return sc, sc64, spec, q, t, rgb_t, d_t


@pytest.mark.parametrize("tile,batch,ppt,graph", [((16, 16), 256, 0, False), ((8, 8), 32, 2, False),
                                                  ((8, 8), 32, 2, True)])
def test_one_keyframe_map_step_matches_oracle(tile, batch, ppt, graph):
    """The benchmark's step (one keyframe: fused projection backward + Adam
    + L_reg) in the default and the benchmark's launch configuration, eager
    and replayed from the captured graph."""
    sc, sc64, spec, q, t, rgb_t, d_t = unit_map_inputs()
    oc = ocam(spec, tile)
    ctx = api.Context(tile=tile, batch=batch, pixels_per_thread=ppt)
    cam = api.camera_from_spec(spec)
    g = api.GaussianParams.from_numpy(sc)
    init = g.clone()
    st = api.AdamMoments(g)
    label = f"map step {tile} {batch} {ppt} {'graph' if graph else 'eager'}"
    flips, excl, _ = gpu_flips(ctx, g, cam, q, t, sc64, oc, label)
    kf = [(api.make_pose(q, t), cu(rgb_t), cu(d_t))]
    cfg = api.MapConfig(use_graph=graph)
    if graph:
        api.map_step(ctx, g, st, cam, kf, None, 1, cfg)  # eager: sizes the scratch for this key
        restore(g, st, init)
    stats = api.map_step(ctx, g, st, cam, kf, None, 1, cfg)
    L, grads = oracle_grads(sc64, [(q, t, rgb_t, d_t, flips)], oc, [1.0], cfg)
    print(label, "loss", stats["loss_last"], "oracle", L)
    assert abs(stats["loss_last"] - L) <= 2e-5 * abs(L)
    assert int(st.step.item()) == 1
    check_first_step(g, st, sc64, grads, cfg, label)
    ctx.close()


def test_map_step_three_iterations_match_oracle():
    """Three one-keyframe iterations (graph-replayed) against three steps of
    the oracle's chain.  The learning rates are scaled by 1e-2 so that the
    parameters whose step direction the gradient bar cannot fix (|g| within
    the bar of 0) move the renders of the next steps by far less than the
    bars; the oracle stores its parameters in float32 after each step, as
    the implementation (and the paper's) does.  The loss of every step, the
    moments after the third and every parameter are compared; a parameter's
    tolerance is the first-order effect of the gradient bar on its three
    Adam steps."""
    sc, sc64, spec, q, t, rgb_t, d_t = unit_map_inputs(7, 8)
    tile = (8, 8)
    oc = ocam(spec, tile)
    ctx = api.Context(tile=tile, batch=32, pixels_per_thread=2)
    cam = api.camera_from_spec(spec)
    g = api.GaussianParams.from_numpy(sc)
    init = g.clone()
    st = api.AdamMoments(g)
    cfg = api.MapConfig(use_graph=True)
    for _, lrk in GROUPS:
        setattr(cfg.adam, lrk, getattr(cfg.adam, lrk) * 1e-2)
    kf = [(api.make_pose(q, t), cu(rgb_t), cu(d_t))]
    api.map_step(ctx, g, st, cam, kf, None, 1, cfg)  # eager sizing run
    restore(g, st, init)
    a = cfg.adam
    P = {k: getattr(sc64, k).copy() for k, _ in GROUPS}
    M = {k: np.zeros_like(P[k]) for k in P}
    V = {k: np.zeros_like(P[k]) for k in P}
    G = []
    for step in (1, 2, 3):
        cur = O.Scene(P["mean"], P["log_scale"], P["quat"], P["opacity_logit"], P["rgb"])
        flips, excl, _ = gpu_flips(ctx, g, cam, q, t, cur, oc, f"three steps, step {step}")
        stats = api.map_step(ctx, g, st, cam, kf, None, 1, cfg)
        L, grads = oracle_grads(cur, [(q, t, rgb_t, d_t, flips)], oc, [1.0], cfg)
        G.append(grads)
        oracle_adam(P, grads, M, V, step, cfg)
        for k in P:  # the parameters are float32 tensors
            P[k] = P[k].astype(np.float32).astype(np.float64)
        print("step", step, "loss", stats["loss_last"], "oracle", L)
        assert abs(stats["loss_last"] - L) <= 2e-5 * abs(L), step
    b1, b2 = a.beta1, a.beta2
    for k, lrk in GROUPS:
        lr = getattr(a, lrk)
        gs = [x[k].reshape(-1) for x in G]
        m_ref, v_ref = M[k].reshape(-1), V[k].reshape(-1)
        m = getattr(st.m, k).cpu().numpy().reshape(-1).astype(np.float64)
        v = getattr(st.v, k).cpu().numpy().reshape(-1).astype(np.float64)
        ok, worst = grad_close(m, m_ref)
        assert ok, (k, "first moment", worst)
        ok, worst = grad_close(np.sqrt(v), np.sqrt(v_ref))
        assert ok, (k, "second moment", worst)
        # first-order bound of the parameter from the gradient bar tol_s of each step:
        # u_t = mh_t / sqrt(vh_t), d u_t / d g_s = a_ts / sqrt(vh_t) - mh_t b_ts g_s / vh_t^1.5
        tol = [1e-3 * (np.abs(x) + 0.1 * np.abs(x).max()) for x in gs]
        bound = np.zeros_like(m_ref)
        for tt in range(3):
            bc1, bc2 = 1 - b1 ** (tt + 1), 1 - b2 ** (tt + 1)
            mh = sum((1 - b1) * b1 ** (tt - s) * gs[s] for s in range(tt + 1)) / bc1
            vh = sum((1 - b2) * b2 ** (tt - s) * gs[s] ** 2 for s in range(tt + 1)) / bc2
            sv = np.sqrt(vh) + a.eps
            for s in range(tt + 1):
                da = (1 - b1) * b1 ** (tt - s) / bc1 / sv
                db = (1 - b2) * b2 ** (tt - s) / bc2 * np.abs(mh * gs[s]) / (sv ** 3)
                bound += np.minimum((da + db) * tol[s], 2.0)
        th = getattr(g, k).detach().cpu().numpy().reshape(-1).astype(np.float64)
        th_ref = P[k].reshape(-1)
        ulp = np.spacing(np.abs(th_ref).astype(np.float32)).astype(np.float64)
        err = np.abs(th - th_ref)
        lim = lr * (np.minimum(bound, 6.0) + 1e-5) + 3 * ulp
        print(k, "worst parameter error / tolerance", (err / lim).max(), "median tolerance / lr",
              np.median(lim) / lr)
        assert (err <= lim).all(), (k, (err / lim).max())
    ctx.close()


@pytest.mark.parametrize("tile,batch,ppt,graph", [((8, 8), 32, 2, True), ((16, 16), 256, 0, False)])
def test_full_size_map_step_matches_oracle(tile, batch, ppt, graph):
    """1200x680 view of the 500k-Gaussian sub-map in the benchmark's launch
    configuration (graph-replayed) and the default one: the loss is
    restricted to a random 2 % of the pixels by giving only those a valid
    target depth (w_color = 0, so the SSIM and colour terms vanish and the
    depth L1 is over the sampled pixels alone), which the oracle's chain can
    follow pixel by pixel; L_reg and Adam still act on all 500k Gaussians."""
    sc = S.room_scene(500_000, seed=3)
    sc64 = O.Scene.from_dict(sc)
    spec = S.camera_room()
    q, t = S.submap_views()[S.HEADLINE_VIEW]
    oc = ocam(spec, tile)
    ctx = api.Context(tile=tile, batch=batch, pixels_per_thread=ppt)
    cam = api.camera_from_spec(spec)
    g = api.GaussianParams.from_numpy(sc)
    init = g.clone()
    st = api.AdamMoments(g)
    label = f"full-size map step {tile} {batch} {ppt}"
    flips, excl, ref = gpu_flips(ctx, g, cam, q, t, sc64, oc, label, max_excluded=1e-3)
    H, W = spec.height, spec.width
    rng = np.random.default_rng(11)
    mask = (rng.random((H, W)) < 0.02) & ~excl & (ref["depth"] > 0.1)
    d_t = np.where(mask, ref["depth"] + np.where(rng.random((H, W)) < 0.5, 0.05, -0.05), 0.0).astype(np.float32)
    rgb_t = np.zeros((3, H, W), np.float32)
    kf = [(api.make_pose(q, t), cu(rgb_t), cu(d_t))]
    cfg = api.MapConfig(use_graph=graph, w_color=0.0)
    if graph:
        api.map_step(ctx, g, st, cam, kf, None, 1, cfg)
        restore(g, st, init)
    stats = api.map_step(ctx, g, st, cam, kf, None, 1, cfg)
    L, grads = oracle_grads(sc64, [(q, t, rgb_t, d_t, flips)], oc, [1.0], cfg)
    print(label, "sampled pixels", mask.sum(), "loss", stats["loss_last"], "oracle", L)
    assert abs(stats["loss_last"] - L) <= 2e-5 * abs(L)
    check_first_step(g, st, sc64, grads, cfg, label)
    ctx.close()


def test_three_keyframe_map_step_matches_oracle():
    """One batched step over three keyframes with weights (0.5, 0.3, 0.2):
    the gradient is the weighted sum of the oracle's per-keyframe gradients
    (Sec. 3.2: the sub-map is optimised over its keyframes jointly)."""
    spec = S.scale_camera(S.camera_room(), 300, 170)
    tile = (16, 16)
    oc = ocam(spec, tile)
    sc_gt = S.room_scene(60_000, seed=3)
    noisy = S.noisy_copy(sc_gt, seed=5)
    sc64 = O.Scene.from_dict(noisy)
    gt64 = O.Scene.from_dict(sc_gt)
    ctx = api.Context(tile=tile)
    cam = api.camera_from_spec(spec)
    g = api.GaussianParams.from_numpy(noisy)
    st = api.AdamMoments(g)
    views, kfs = [], []
    for i in (1, 4, 6):
        q, t = S.submap_views()[i]
        flips, excl, r = gpu_flips(ctx, g, cam, q, t, sc64, oc, f"keyframe {i}")
        tg = O.render(gt64, q, t, oc)
        rgb_t, d_t = margin_target(r["rgb"], r["depth"], tg["rgb"], tg["depth"])
        views.append((q, t, rgb_t, d_t, flips))
        kfs.append((api.make_pose(q, t), cu(rgb_t), cu(d_t)))
    w = [0.5, 0.3, 0.2]
    cfg = api.MapConfig(use_graph=False)
    stats = api.map_step(ctx, g, st, cam, kfs, w, 1, cfg)
    L, grads = oracle_grads(sc64, views, oc, w, cfg)
    print("three keyframes: loss", stats["loss_last"], "oracle", L)
    assert abs(stats["loss_last"] - L) <= 2e-5 * abs(L)
    check_first_step(g, st, sc64, grads, cfg, "three keyframes")
    ctx.close()
