"""The learned warm-start, trained on the GPU on synthetic rooms, reduces the
error of a perturbed initial pose on held-out rooms, and the warm-started
tracker (falling back to the plain initial pose when the network's pose has
the larger tracking loss) needs no more iterations and fewer wall-clock ms
per frame than the plain one, network and fallback test included.

Training rooms: room_scene(200k Gaussians), seeds 1000-1095, 24 frames each
(trajectories with about 4 cm / 3 degrees between frames), 32 initial poses
per frame (73728 samples, 45 GB of inputs on the device); initial pose = true
pose moved by a random twist of up to 5 cm / 3 degrees; 6000 Adam steps of
256.  Held-out rooms: seeds 2000-2002, 16 frames x 4 initial poses.
"""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_2312_10070_gb300 import api, synth
    from paper_2312_10070_gb300 import warmstart as W
    spec = synth.camera_room()
    ctx_f = api.Context(tile=(16, 16), batch=256)
    ctx_l = api.Context(tile=(16, 16), batch=64)
    rng = np.random.default_rng(5)
    n_rooms, frames, per_frame = 96, 24, 32
    train = W.Samples(n_rooms * frames * per_frame, seed=1)
    for r in range(n_rooms):
        seed = 1000 + r
        g = api.GaussianParams.from_numpy(synth.room_scene(200_000, seed=seed))
        poses = synth.room_trajectory(seed=seed, n_frames=frames, step_m=0.04, max_step_deg=3.0)
        W.add_frames(train, ctx_f, ctx_l, g, spec, poses, per_frame, rng, noise_seed=10 * seed, keep_frames=False)
    evals = []
    for seed in (2000, 2001, 2002):
        g = api.GaussianParams.from_numpy(synth.room_scene(200_000, seed=seed))
        poses = synth.room_trajectory(seed=seed, n_frames=16, step_m=0.04, max_step_deg=3.0)
        ev = W.Samples(16 * 4, seed=seed)
        W.add_frames(ev, ctx_f, ctx_l, g, spec, poses, 4, np.random.default_rng(seed), noise_seed=10 * seed)
        evals.append((g, ev))
    net = W.WarmStartNet(max_batch=256, seed=7)
    losses = W.train(net, train, steps=6000, batch=256, lr=5e-4, seed=8, log_every=500)
    return dict(W=W, api=api, spec=spec, ctx_f=ctx_f, ctx_l=ctx_l, net=net, evals=evals, losses=losses)


def test_training_loss_decreases(trained):
    losses = trained["losses"]
    assert losses[-1][1] < 0.5 * losses[0][1], losses


def test_warm_start_reduces_held_out_pose_error(trained):
    W, net = trained["W"], trained["net"]
    m0, m1 = [], []
    for _, ev in trained["evals"]:
        pred = W.predict(net, ev.x)
        m0.append(np.median(W.pose_errors(ev, ev.init), axis=0))
        m1.append(np.median(W.pose_errors(ev, W.corrected_poses(ev, pred)), axis=0))
    m0, m1 = np.mean(m0, axis=0), np.mean(m1, axis=0)
    print("median init error (m, deg)", m0, "after warm start", m1)
    assert m1[0] < 0.85 * m0[0] and m1[1] < 0.85 * m0[1], (m0, m1)


def _wall_ms(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, (time.perf_counter() - t0) * 1e3


def test_warm_started_tracker_with_fallback(trained):
    """Iterations and wall-clock ms per frame to reach 1 cm / 0.5 degrees,
    plain against warm-started, on the three held-out rooms x 8 frames.  The
    warm-started frame pays for the network (160 x 120 render, input builder,
    batch-1 forward, twist applied on the device and read back), for the
    fallback test (tracking loss at both start poses, one tracker iteration
    each) and for its own tracker iterations; the plain frame for its tracker
    iterations only.  Every frame's graphs are captured before the timed
    calls (the convergence search runs first on the same frame).  The
    warm-started tracker must need fewer wall-clock ms per frame on average,
    and no more iterations."""
    W, net = trained["W"], trained["net"]
    ctx_f, ctx_l, spec = trained["ctx_f"], trained["ctx_l"], trained["spec"]
    budgets = (10, 20, 40, 80, 160)
    cap = 2 * budgets[-1]
    plain, warm, fallbacks, plain_ms, warm_ms, room_ms = [], [], 0, [], [], []
    for room, (g, ev) in enumerate(trained["evals"]):
        r0 = len(plain_ms)
        for k in range(0, 24, 3):
            fr = ev.frames[ev.frame[k]]
            q0, t0 = ev.init[k]
            n0, loss0, _ = W.iterations_to_converge(ctx_f, g, spec, fr, q0, t0, budgets)
            qw, tw = W.warm_start_pose(net, ctx_l, g, spec, fr, q0, t0)
            n1, loss1, _ = W.iterations_to_converge(ctx_f, g, spec, fr, qw, tw, budgets)
            use_warm = loss1 <= loss0
            if not use_warm:  # fallback: keep the plain initial pose
                n1, fallbacks = n0, fallbacks + 1
            plain.append(n0 if n0 is not None else cap)
            warm.append(n1 if n1 is not None else cap)
            # wall clock of each path for this frame
            _, ms0 = _wall_ms(lambda: W.track_from(ctx_f, g, spec, fr, q0, t0, plain[-1]))
            (qw2, tw2), ms_net = _wall_ms(lambda: W.warm_start_pose(net, ctx_l, g, spec, fr, q0, t0))
            _, ms_check = _wall_ms(lambda: (W.track_from(ctx_f, g, spec, fr, qw2, tw2, 1),
                                            W.track_from(ctx_f, g, spec, fr, q0, t0, 1)))
            qs, ts = (qw2, tw2) if use_warm else (q0, t0)
            _, ms1 = _wall_ms(lambda: W.track_from(ctx_f, g, spec, fr, qs, ts, warm[-1]))
            plain_ms.append(ms0)
            warm_ms.append(ms_net + ms_check + ms1)
        room_ms.append((float(np.mean(plain_ms[r0:])), float(np.mean(warm_ms[r0:]))))
    print("iterations plain", plain, "warm", warm, "fallbacks", fallbacks)
    print("ms per frame plain %.2f warm-started %.2f; per room (plain, warm) %s"
          % (np.mean(plain_ms), np.mean(warm_ms), np.round(room_ms, 2).tolist()))
    assert np.mean(warm) <= np.mean(plain), (np.mean(warm), np.mean(plain))
    assert np.mean(warm_ms) < np.mean(plain_ms), (np.mean(warm_ms), np.mean(plain_ms))
