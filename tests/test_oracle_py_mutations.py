"""The pins of the Python oracles (oracle/cnn.py: the warm-start network;
oracle/seed.py: sub-map seeding) catch plausible mistakes.  Each case copies
the oracle package and the module's pin file into a temporary tree, plants
one mistake in the copy (a dropped mask or factor, a transposed kernel, an
overwrite instead of an accumulation, a wrong constant, sign or offset), and
runs the pins there in a subprocess: at least one must fail.  The unmodified
copy must pass them all.  CPU only."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the mistake is, oracle module, pin file, text, replacement)
MUTATIONS = [
    ("cnn: 3x3 taps transposed in im2col", "cnn.py", "test_oracle_cnn_pins.py",
     "cols[:, :, :, ky, kx, :] = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :]",
     "cols[:, :, :, kx, ky, :] = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :]"),
    ("cnn: col2im overwrites instead of accumulating", "cnn.py", "test_oracle_cnn_pins.py",
     "dxp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :] += d[:, :, :, ky, kx, :]",
     "dxp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :] = d[:, :, :, ky, kx, :]"),
    ("cnn: ReLU mask of the dense layer dropped in the backward", "cnn.py", "test_oracle_cnn_pins.py",
     "dz1 = rnd(dh1 * (z1 > 0))", "dz1 = rnd(dh1)"),
    ("cnn: output bias gradient averaged over the batch", "cnn.py", "test_oracle_cnn_pins.py",
     'g["fc1.b"] = d_out.sum(0)', 'g["fc1.b"] = d_out.mean(0)'),
    ("cnn: factor 2 of the squared error's derivative dropped", "cnn.py", "test_oracle_cnn_pins.py",
     "return float(np.sum(w * r * r) / B), 2.0 * w * r / B", "return float(np.sum(w * r * r) / B), w * r / B"),
    ("cnn: invalid depth averaged in the box downsample", "cnn.py", "test_oracle_cnn_pins.py",
     "out_d[i, j] = dv[m].mean() if m.any() else 0.0", "out_d[i, j] = dv.mean()"),
    ("cnn: depth residual kept where the frame's depth is invalid", "cnn.py", "test_oracle_cnn_pins.py",
     "valid = (d_r > 0) & (d_i > 0)", "valid = d_r > 0"),
    ("cnn: rendered depth channel not scaled", "cnn.py", "test_oracle_cnn_pins.py",
     "ch = [rgb_r[0], rgb_r[1], rgb_r[2], d_r / depth_scale,", "ch = [rgb_r[0], rgb_r[1], rgb_r[2], d_r,"),
    ("seed: prune by sigmoid(-logit)", "seed.py", "test_oracle_seed_pins.py",
     'o = 1.0 / (1.0 + np.exp(-np.asarray(params["opacity_logit"], np.float64)))',
     'o = 1.0 / (1.0 + np.exp(np.asarray(params["opacity_logit"], np.float64)))'),
    ("seed: splitmix64 first multiplier", "seed.py", "test_oracle_seed_pins.py",
     "z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)",
     "z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B7)"),
    ("seed: largest keys sampled instead of smallest", "seed.py", "test_oracle_seed_pins.py",
     "order = np.lexsort((cand, keys[cand]))  # by key, then pixel index",
     "order = np.lexsort((cand, -keys[cand].astype(np.int64)))"),
    ("seed: one-sided difference in the colour gradient", "seed.py", "test_oracle_seed_pins.py",
     "gx = (y[1:-1, 2:] - y[1:-1, :-2]) / 2.0", "gx = (y[1:-1, 2:] - y[1:-1, 1:-1]) / 2.0"),
    ("seed: back-projection without the pixel-centre offset", "seed.py", "test_oracle_seed_pins.py",
     "pc = np.stack([(j + 0.5 - cam.cx) * z / cam.fx, (i + 0.5 - cam.cy) * z / cam.fy, z], axis=1)",
     "pc = np.stack([(j - cam.cx) * z / cam.fx, (i - cam.cy) * z / cam.fy, z], axis=1)"),
    ("seed: camera-to-world with R instead of R^T", "seed.py", "test_oracle_seed_pins.py",
     "return (pc - np.asarray(t, np.float64)) @ R  # rows: R^T (p_c - t)",
     "return (pc - np.asarray(t, np.float64)) @ R.T"),
    ("seed: nearest neighbour includes the point itself", "seed.py", "test_oracle_seed_pins.py",
     "                d[np.nonzero(hit)[0], r[hit] - p0] = np.inf", "                pass"),
    ("seed: merge radius 2 rho", "seed.py", "test_oracle_seed_pins.py",
     "        add = d2 >= rho * rho", "        add = d2 >= 4 * rho * rho"),
]


def make_tree(d, module=None, old=None, new=None):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    os.makedirs(os.path.join(d, "tests"))
    for f in ("__init__.py", "conftest.py", "test_oracle_cnn_pins.py", "test_oracle_seed_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    if module:
        p = os.path.join(d, "oracle", module)
        src = open(p).read()
        assert src.count(old) == 1, f"mutation site not unique or missing: {old}"
        open(p, "w").write(src.replace(old, new))
    return d


def run_pins(d, pin_file):
    env = dict(os.environ, OMP_NUM_THREADS="2", OPENBLAS_NUM_THREADS="2", MKL_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", pin_file), "-x", "-q",
                        "-p", "no:cacheprovider"], capture_output=True, text=True, cwd=d, env=env, timeout=600)
    return r.returncode, r.stdout[-1500:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    jobs = []
    for pin in ("test_oracle_cnn_pins.py", "test_oracle_seed_pins.py"):
        jobs.append((f"unmodified {pin}", make_tree(str(tmp_path_factory.mktemp("orig"))), pin))
    for name, module, pin, old, new in MUTATIONS:
        jobs.append((name, make_tree(str(tmp_path_factory.mktemp("mut")), module, old, new), pin))
    with ThreadPoolExecutor(max_workers=4) as ex:
        out = list(ex.map(lambda j: run_pins(j[1], j[2]), jobs))
    return {j[0]: o for j, o in zip(jobs, out)}


@pytest.mark.parametrize("pin", ["test_oracle_cnn_pins.py", "test_oracle_seed_pins.py"])
def test_unmodified_copy_passes_every_pin(results, pin):
    rc, out = results[f"unmodified {pin}"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(results, name):
    rc, out = results[name]
    assert rc != 0, f"no pin caught: {name}\n{out}"
