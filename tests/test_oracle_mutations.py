"""Mutation check of the oracle's pins.

Each entry plants one plausible mistake in a copy of ``oracle/`` (a dropped
term, a wrong sign or index, a transposed operand, a wrong constant) and runs
the oracle's CPU pins against the mutated copy; at least one pin must fail.
An unmutated copy must pass, so a failure is the mutation's doing and not the
harness's.  This is what makes the pins evidence: an oracle mistake that no
pin notices would be carried into every GPU parity claim.

The copies live in a temporary directory (oracle/, tests/ and the package's
Python files); nothing in the repository is modified.  The C oracle of each
copy is compiled inside it.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_variants.py", "tests/test_oracle_loss.py",
        "tests/test_oracle_relocation.py", "tests/test_oracle_window.py"]

C = "oracle/sss_oracle.c"
LOSS = "oracle/image_loss.py"
RELOC = "oracle/relocation.py"

# (name, file, original text, planted text); the original must occur exactly once
MUTATIONS = [
    ("2D exponent -(nu+3)/2 instead of -(nu+2)/2", C,
     "return pow(1.0 + h / nu, -(nu + 2.0) / 2.0); }", "return pow(1.0 + h / nu, -(nu + 3.0) / 2.0); }"),
    ("conic off-diagonal sign", C, "out[G_CB] = -cov[1] / det;", "out[G_CB] = cov[1] / det;"),
    ("h without the 2 of 2 b dx dy", C,
     "return r[P_CON_A] * dx * dx + 2.0 * r[P_CON_B] * dx * dy", "return r[P_CON_A] * dx * dx + r[P_CON_B] * dx * dy"),
    ("J W^T instead of J W", C,
     "A[r * 3 + c] = J[r * 3 + 0] * V[0 * 4 + c] + J[r * 3 + 1] * V[1 * 4 + c] + J[r * 3 + 2] * V[2 * 4 + c]",
     "A[r * 3 + c] = J[r * 3 + 0] * V[c * 4 + 0] + J[r * 3 + 1] * V[c * 4 + 1] + J[r * 3 + 2] * V[c * 4 + 2]"),
    ("dT/dh sign", C, "return -(nu + 2.0) / (2.0 * nu) * pow(1.0 + h / nu, -(nu + 4.0) / 2.0); }",
     "return (nu + 2.0) / (2.0 * nu) * pow(1.0 + h / nu, -(nu + 4.0) / 2.0); }"),
    ("dC/dalpha without the (1 - alpha) division", C,
     "double dC_dalpha = c->T * r[P_R + ch] - (S[ch] + T_final * cfg->bg[ch]) / (1.0 - c->alpha);",
     "double dC_dalpha = c->T * r[P_R + ch] - (S[ch] + T_final * cfg->bg[ch]);"),
    ("quaternion cross-term sign", C, "{1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z),",
     "{1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y + w * z),"),
    ("SH without the Condon-Shortley phase", C, "qmm *= -(2.0 * k - 1.0);", "qmm *= (2.0 * k - 1.0);"),
    ("SH colour without the +0.5 offset", C, "cx acc = 0.5;", "cx acc = 0.0;"),
    ("SGHMC momentum without friction", C, "double r_new = (1.0 - eps * C) * rr - eps * G + sq * xi[c];",
     "double r_new = rr - eps * G + sq * xi[c];"),
    ("SGHMC noise scale sqrt(2 C) instead of sqrt(2 eps C)", C, "double sq = sqrt(2.0 * eps * C);",
     "double sq = sqrt(2.0 * C);"),
    ("Adam without bias corrections", C, "theta[j] -= lr * (mm / bc1) / (sqrt(vv / bc2) + aeps);",
     "theta[j] -= lr * mm / (sqrt(vv) + aeps);"),
    ("Adam first moment from v", C, "double mm = b1 * m[j] + (1.0 - b1) * gg;",
     "double mm = b1 * v[j] + (1.0 - b1) * gg;"),
    ("Adam second moment without the square", C, "double vv = b2 * v[j] + (1.0 - b2) * gg * gg;",
     "double vv = b2 * v[j] + (1.0 - b2) * fabs(gg);"),
    ("burn-in Sigma as R^T D R", C, "sig += R[a * 3 + k] * s2[k] * R[b * 3 + k];",
     "sig += R[k * 3 + a] * s2[k] * R[k * 3 + b];"),
    ("burn-in keeps the friction term", C, "if (burn_in) mu += g * eps * sq * noise[c];",
     "if (burn_in) mu += g * eps * (1.0 - eps * C) * rr + g * eps * sq * noise[c];"),
    ("gate on signed o", C, "double g = 1.0 / (1.0 + exp(kk * (fabs(o) - t0)));",
     "double g = 1.0 / (1.0 + exp(kk * (o - t0)));"),
    ("termination after the splat instead of before", C,
     "int term = Tn < cfg->t_min;", "int term = T < cfg->t_min;"),
    ("an ambiguous alpha decision that cannot be flipped", C,
     "if (ev < 32 && ((flip >> ev) & 1u)) include = !include;", ""),
    ("an ambiguous termination that cannot be flipped", C,
     "if (ev < 32 && ((flip >> ev) & 1u)) term = !term;", ""),
    ("no lower alpha clamp", C, "if (alpha < -cfg->alpha_max) { alpha = -cfg->alpha_max; clamped = 1; }", ""),
    ("Philox key constant", C, "k0 += 0x9E3779B9u;", "k0 += 0x9E3779BBu;"),
    ("Box-Muller second normal as cos", C, "z[1] = r1 * sin(2.0 * ORC_PI * u2);",
     "z[1] = r1 * cos(2.0 * ORC_PI * u2);"),
    ("fx for the y coordinate", C, "out[G_MY] = cam->fy * p[1] / p[2] + cam->cy;",
     "out[G_MY] = cam->fx * p[1] / p[2] + cam->cy;"),
    ("back-to-front order", C, "if (x->depth < y->depth) return -1;\n  if (x->depth > y->depth) return 1;",
     "if (x->depth < y->depth) return 1;\n  if (x->depth > y->depth) return -1;"),
    ("exact dT/dnu without its log term", C,
     "return -0.5 * log1p(h / nu) * pow(g, -(nu + 2.0) / 2.0) + second;", "return second;"),
    ("nu limited at 1e3", C, "((nur > 1e4) ? (cx)1e4 : nu_in)", "((nur > 1e3) ? (cx)1e3 : nu_in)"),
    ("extent from sqrt(cov) h_max", C, "double ex = sqrt(rec[P_COV_A] * hmax)", "double ex = sqrt(rec[P_COV_A]) * hmax"),
    ("Gaussian kernel exp(-h)", C, "return cfg->kernel == 1 ? exp(-0.5 * h) : orc_t2d(h, nu);",
     "return cfg->kernel == 1 ? exp(-h) : orc_t2d(h, nu);"),
    ("SSIM C2 = 0.03", LOSS, "C2 = 0.03 ** 2", "C2 = 0.03"),
    ("SSIM sigma_xy without the mean product", LOSS,
     "        sxy = window_sum(xc * yc, w) - mx * my\n        out[c]", "        sxy = window_sum(xc * yc, w)\n        out[c]"),
    ("SSIM gradient without the 2 x (w * b) term", LOSS,
     "g[c] = window_sum(a, w) + 2 * xc * window_sum(dS_dsx2, w) + yc * window_sum(dS_dsxy, w)",
     "g[c] = window_sum(a, w) + yc * window_sum(dS_dsxy, w)"),
    ("opacity regulariser gradient without 1 - o^2", LOSS, "eps_o * np.sign(o) * (1.0 - o * o)", "eps_o * np.sign(o)"),
    ("relocated opacity without the N-th root", RELOC, "a = 1.0 - (1.0 - abs(o_old)) ** (1.0 / N)",
     "a = 1.0 - (1.0 - abs(o_old)) / N"),
    ("relocation K without the alternating sign", RELOC, "math.comb(i - 1, k) * (-1) ** k * o ** (k + 1)",
     "math.comb(i - 1, k) * o ** (k + 1)"),
    ("relocation Beta argument nu + 2 instead of nu + 3", RELOC,
     "beta(0.5, ((k + 1) * (nu_new + 3.0) - 1.0) / 2.0)", "beta(0.5, ((k + 1) * (nu_new + 2.0) - 1.0) / 2.0)"),
    ("relocation draw from the prefix's left side", RELOC, "np.searchsorted(prefix, v, side=\"right\")",
     "np.searchsorted(prefix, v, side=\"left\")"),
    # the ambiguity window must bound an FP32 evaluation of alpha
    ("window without the FP32 evaluation of h", C, "gm + 7.0 * u * q;", "gm + 1.0 * u * q;"),
    ("window without the FP32 scales", C, "const double dh = 8.0 * u * h + ", "const double dh = "),
    ("window without the argument 1 + h/nu", C, "ORC_MUFU + 3.0 * u * e + 2.0 * u * e", "ORC_MUFU + 2.0 * u * e"),
    ("window without the opacity", C, "  w += 5.0 * u;\n", "  w += 0.0 * u;\n"),
    ("window without the log2 error", C, "log(2.0) * e * ORC_MUFU + 3.0", "3.0"),
    ("window without the h error", C, "w = e / nu / (1.0 + h / nu) * dh + ", "w = "),
    ("Gaussian window without dlnT2D/dh", C, "w = 0.5 * dh + ORC_MUFU + u * h;", "w = ORC_MUFU + u * h;"),
    # the termination window must bound an FP32 compositing of T
    ("T bound without the 2u roundings", C, "errT + 2.0 * ORC_U + W * fabs(alpha)", "errT + W * fabs(alpha)"),
    ("T bound without the alpha error", C, "errT + 2.0 * ORC_U + W * fabs(alpha) / fabs(1.0 - alpha);",
     "errT + 2.0 * ORC_U;"),
    ("T bound with alpha / (1 + alpha)", C, "W * fabs(alpha) / fabs(1.0 - alpha);", "W * fabs(alpha) / fabs(1.0 + alpha);"),
    ("T bound not accumulated", C, "double errTn = errT + 2.0 * ORC_U", "double errTn = 2.0 * ORC_U"),
]


def _copy_tree(dst):
    ign = shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.o", ".pytest_cache")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"), ignore=ign)
    pkg = os.path.join(dst, "paper_2503_10148_gb300")
    os.makedirs(pkg)
    for f in os.listdir(os.path.join(ROOT, "paper_2503_10148_gb300")):
        if f.endswith(".py"):
            shutil.copy(os.path.join(ROOT, "paper_2503_10148_gb300", f), pkg)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)


def _run_pins(dst):
    b = subprocess.run([sys.executable, "oracle/build.py", "--force"], cwd=dst, capture_output=True, text=True,
                       timeout=300)
    if b.returncode != 0:
        return "build", b.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider"], cwd=dst,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-3000:]


def _mutant(i):
    name, path, old, new = MUTATIONS[i]
    with tempfile.TemporaryDirectory(prefix="orc_mut_") as d:
        _copy_tree(d)
        p = os.path.join(d, path)
        with open(p) as f:
            src = f.read()
        assert src.count(old) == 1, f"{name}: original text found {src.count(old)} times in {path}"
        with open(p, "w") as f:
            f.write(src.replace(old, new))
        return _run_pins(d)


def test_unmutated_copy_passes_every_pin():
    with tempfile.TemporaryDirectory(prefix="orc_mut_") as d:
        _copy_tree(d)
        rc, out = _run_pins(d)
    assert rc == 0, out


def test_every_planted_mistake_fails_a_pin():
    workers = min(8, os.cpu_count() or 2)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(_mutant, range(len(MUTATIONS))))
    survived = []
    for (name, path, _, _), (rc, out) in zip(MUTATIONS, results):
        assert rc != "build", f"{name}: mutated oracle did not compile:\n{out}"
        # pytest exit code 1 = tests ran and at least one failed
        if rc != 1 or "failed" not in out:
            survived.append(f"{name} ({path}): pytest rc {rc}")
    assert not survived, "mutations no pin detects:\n" + "\n".join(survived)
