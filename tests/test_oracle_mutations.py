"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of oracle/gsr_oracle.c (a flipped sign, a dropped term, a
transposed operand, a swapped index, a wrong constant or threshold), builds
it, and runs the CPU pin tests (tests/test_oracle_pins.py) against that
build in a subprocess: at least one pin must fail.  The unmodified copy,
built the same way, must pass them all, so each failure is the planted
mistake's.  Nothing here touches a GPU or the CUDA path."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gsr_oracle.c")

# (what the mistake is, text in gsr_oracle.c, its replacement); a mistake that
# spans several sites gives tuples of texts and replacements
MUTATIONS = [
    ("pose adjoint: sign of the rotation term from Sigma_cam",
     "g_pose[3] += 2.0 * (Y[7] - Y[5]);", "g_pose[3] += 2.0 * (Y[5] - Y[7]);"),
    ("pose adjoint: rotation part of the point term",
     "g_pose[4] = pz * gp[0] - px * gp[2];", "g_pose[4] = px * gp[2] - pz * gp[0];"),
    ("depth gradient: direct route dD/dz = alpha T dropped",
     "gp[2] += g2[9];", "gp[2] += 0.0 * g2[9];"),
    ("opacity: sigmoid derivative dropped",
     "*g_logit = g2[5] * o->opacity * (1.0 - o->opacity);", "*g_logit = g2[5] * o->opacity;"),
    ("camera transform: rotation transposed",
     "o->p[i] = Rcw[3 * i] * mean[0] + Rcw[3 * i + 1] * mean[1] + Rcw[3 * i + 2] * mean[2] + tcw[i];",
     "o->p[i] = Rcw[i] * mean[0] + Rcw[3 + i] * mean[1] + Rcw[6 + i] * mean[2] + tcw[i];"),
    ("conic: diagonal entries swapped",
     "o->conic[0] = cc / det; o->conic[1] = -b / det; o->conic[2] = a / det;",
     "o->conic[0] = a / det; o->conic[1] = -b / det; o->conic[2] = cc / det;"),
    ("EWA: J's x/z coupling sign",
     "J[0] = c->fx / pz; J[1] = 0; J[2] = -c->fx * tx / pz;", "J[0] = c->fx / pz; J[1] = 0; J[2] = c->fx * tx / pz;"),
    ("low-pass dilation dropped from the first diagonal entry",
     "double a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + c->eps2d;",
     "double a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2];"),
    ("pixel centre at the corner", "double px = ix + 0.5, py = iy + 0.5;", "double px = ix, py = iy;"),
    ("alpha cap 0.999", "#define ALPHA_MAX 0.99", "#define ALPHA_MAX 0.999"),
    ("transmittance stop after compositing", "int stop = Tn < T_STOP;", "int stop = T < T_STOP;"),
    ("blend adjoint: suffix sum not divided by 1 - alpha",
     "for (int ch = 0; ch < 3; ++ch) dLda += dC[ch] * (cj[ch] * e->T - Sc[ch] / om);",
     "for (int ch = 0; ch < 3; ++ch) dLda += dC[ch] * (cj[ch] * e->T - Sc[ch]);"),
    ("SSIM: C2 = C1", "const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;",
     "const double C1 = 0.01 * 0.01, C2 = 0.01 * 0.01;"),
    ("tracking: upper instead of lower median", "med = e[(nv - 1) / 2];", "med = e[nv / 2];"),
    ("L_reg: scale mean over two axes", "sb /= 3.0;", "sb /= 2.0;"),
    ("Adam: second-moment bias correction dropped", "double mh = m1[i] / bc1, vh = m2[i] / bc2;",
     "double mh = m1[i] / bc1, vh = m2[i];"),
    ("tile rectangle: right edge one tile short", "o->x1 = imin(tiles_x - 1, (int)floor(ex[1] / c->tile_w));",
     "o->x1 = imin(tiles_x - 1, (int)floor(ex[1] / c->tile_w) - 1);"),
    ("sort: depth order reversed", "if (da < db) return -1;\n    if (da > db) return 1;",
     "if (da < db) return 1;\n    if (da > db) return -1;"),
    ("log-scale chain: ds/dlog s = s dropped", "g_ls[k] = gs * o->s[k];", "g_ls[k] = gs;"),
    ("quaternion: normalisation's projection dropped",
     "for (int k = 0; k < 4; ++k) g_quat[k] = (gqh[k] - o->qhat[k] * dot) / o->qnorm;",
     "for (int k = 0; k < 4; ++k) g_quat[k] = gqh[k] / o->qnorm;"),
    ("SE(3) retraction: V's second-order term dropped", "V[i] = I + B * K[i] + Cc * K2[i];",
     "V[i] = I + B * K[i];"),
    ("tracking: colour residual weighted by 1 - lambda_c",
     "L += w * (lam_c * lc + (1 - lam_c) * ed);", "L += w * ((1 - lam_c) * lc + (1 - lam_c) * ed);"),
    ("tracking: alpha mask with exponent 1", "double w = in ? pow(alpha[p], apow) : 0.0;",
     "double w = in ? alpha[p] : 0.0;"),
    ("alpha skip threshold 1/128", "#define ALPHA_MIN (1.0 / 255.0)", "#define ALPHA_MIN (1.0 / 128.0)"),
    ("transmittance stop threshold 1e-3", "#define T_STOP 1e-4", "#define T_STOP 1e-3"),
    ("SSIM window sigma 2", "exp(-((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5))",
     "exp(-((k - 5) * (k - 5)) / (2.0 * 2.0 * 2.0))"),
    ("depth L1 over invalid pixels too",
     ("if (depth_t[p] > 0) { ++nvalid; l1d += fabs(depth[p] - depth_t[p]); }",
      "d_depth[p] = (depth_t[p] > 0 && nvalid > 0)"),
     ("if (depth_t[p] >= 0) { ++nvalid; l1d += fabs(depth[p] - depth_t[p]); }",
      "d_depth[p] = (depth_t[p] >= 0 && nvalid > 0)")),
    ("opacity: sigmoid of -logit", "o->opacity = 1.0 / (1.0 + exp(-logit));", "o->opacity = 1.0 / (1.0 + exp(logit));"),
    ("quaternion: sign of w z in R[0][1]", "R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);",
     "R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y + w * z);"),
    ("backward: sign of the conic inverse's derivative",
     "GS[2 * i + j] = -(T2[2 * i] * Q[j] + T2[2 * i + 1] * Q[2 + j]);",
     "GS[2 * i + j] = (T2[2 * i] * Q[j] + T2[2 * i + 1] * Q[2 + j]);"),
    ("backward: factor 2 of dL/dJ dropped",
     "GJ[3 * r + k] = 2.0 * (GS[2 * r] * JSc[k] + GS[2 * r + 1] * JSc[3 + k]);",
     "GJ[3 * r + k] = (GS[2 * r] * JSc[k] + GS[2 * r + 1] * JSc[3 + k]);"),
    ("backward: off-diagonal conic gradient not halved", "double GQ[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};",
     "double GQ[4] = {g2[2], g2[3], g2[3], g2[4]};"),
    ("pose adjoint: sign of the z-rotation term from Sigma_cam", "g_pose[5] += 2.0 * (Y[3] - Y[1]);",
     "g_pose[5] += 2.0 * (Y[1] - Y[3]);"),
    ("backward: factor 2 of dL/dM dropped", "for (int i = 0; i < 9; ++i) GM[i] *= 2.0;",
     "for (int i = 0; i < 9; ++i) GM[i] *= 1.0;"),
    ("backward: sign of dJ00/dz", "gp[2] += GJ[0] * (-fx / (pz * pz)) + GJ[2] * (fx * o->tx / (pz * pz))",
     "gp[2] += GJ[0] * (fx / (pz * pz)) + GJ[2] * (fx * o->tx / (pz * pz))"),
    ("near plane at the camera centre",
     ("if (pz <= c->z_near && !z_amb) return;", "if (empty || pz <= c->z_near) return;"),
     ("if (pz <= 0.0 && !z_amb) return;", "if (empty || pz <= 0.0) return;")),
    ("SE(3) left Jacobian: sign of the second coupling coefficient",
     "c2 = (t2 + 2 * cos(th) - 2) / (2 * t2 * t2);", "c2 = -(t2 + 2 * cos(th) - 2) / (2 * t2 * t2);"),
    ("SE(3) left Jacobian: coupling block transposed", "J[6 * r + (c + 3)] = Q;",
     "J[6 * c + (r + 3)] = Q;"),
    ("guard band: gradient through the clamped coordinate",
     "if (!o->clamp_x) { gp[0] += gtx / pz; gp[2] += -gtx * px / (pz * pz); }",
     "{ gp[0] += gtx / pz; gp[2] += -gtx * px / (pz * pz); }"),
]


def build(text, path):
    c = path + ".c"
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", path, c, "-lm"])
    return path


def run_pins(lib):
    env = dict(os.environ, GSR_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x",
                        "-q", "-p", "no:cacheprovider", "-m", "not gpu"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=600)
    return r.returncode, r.stdout[-1500:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("mutants"))
    src = open(SRC).read()
    texts = [("unmodified", src)]
    for name, old, new in MUTATIONS:
        olds, news = (old, new) if isinstance(old, tuple) else ((old,), (new,))
        text = src
        for o, n in zip(olds, news):  # a mistake may span several sites
            assert text.count(o) == 1, f"mutation site not unique or missing: {name}"
            text = text.replace(o, n)
        texts.append((name, text))
    libs = [build(t, os.path.join(d, f"m{i}.so")) for i, (_, t) in enumerate(texts)]
    with ThreadPoolExecutor(max_workers=4) as ex:
        out = list(ex.map(run_pins, libs))
    return {name: o for (name, _), o in zip(texts, out)}


def test_unmodified_copy_passes_every_pin(results):
    rc, out = results["unmodified"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(results, name):
    rc, out = results[name]
    assert rc != 0, f"no pin caught: {name}\n{out}"
