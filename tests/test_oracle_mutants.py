"""Planted mistakes in the oracle, on the CPU, to show that its pins catch them.

Each mutant is gl_oracle.cpp with one plausible error (a dropped term, a wrong
sign, a wrong power or index, transposed operands), compiled under
oracle/_build/mutants/. The oracle's pin tests (closed forms, library
routines, invariants and brute force) then run against it in a subprocess.
Every mutant must fail at least one pin, and the unmodified source, built and
run the same way, must pass them all."""
import concurrent.futures
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gl_oracle.cpp")
OUT = os.path.join(ROOT, "oracle", "_build", "mutants")
PINS = ["tests/test_oracle_epl.py", "tests/test_oracle_light.py", "tests/test_oracle_image.py",
        "tests/test_oracle_likelihood.py"]
MUTANTS = [
    ("series ratio sign", "T ratio = -f * (2.0 * n - (2.0 - t))", "T ratio = f * (2.0 * n - (2.0 - t))"),
    ("series ratio denominator", "/ (2.0 * n + (2.0 - t));", "/ (2.0 * n + 1.0);"),
    ("series term power", "term = cmul(term, e2iv);", "term = cmul(term, eiv);"),
    ("EPL radial power", "pow(b / R, t - 1.0)", "pow(b / R, t)"),
    ("EPL elliptical radius", "sqrt(q * q * xp * xp + yp * yp)", "sqrt(q * xp * xp + yp * yp)"),
    ("EPL scale radius", "T b = p[0] * sqrt(q);", "T b = p[0];"),
    ("EPL rotation back sign", "ax = cs * alr - sn * ali;", "ax = cs * alr + sn * ali;"),
    ("EPL angle operand", "Cx<T> eiv = {q * xp / R, yp / R};", "Cx<T> eiv = {xp / R, q * yp / R};"),
    ("axis ratio", "q = (1.0 - c) / (1.0 + c);", "q = 1.0 - c;"),
    ("position angle operands", "phi = 0.5 * atan2(e2, e1);", "phi = 0.5 * atan2(e1, e2);"),
    ("shear sign", "T by = y - ay - (g2 * x - g1 * y);", "T by = y - ay - (g2 * x + g1 * y);"),
    ("source plane drops deflection", "T bx = x - ax - (g1 * x + g2 * y);", "T bx = x - (g1 * x + g2 * y);"),
    ("Sersic axes transposed", "sqrt(q * xp * xp + yp * yp / q)", "sqrt(xp * xp / q + q * yp * yp)"),
    ("Sersic b_n sign", "1.9992 * p[1] - 0.3271", "1.9992 * p[1] + 0.3271"),
    ("Sersic exponent", "pow(R / p[0], 1.0 / p[1])", "pow(R / p[0], p[1])"),
    ("Sersic frame rotation sign", "  T yp = -sn * dx + cs * dy;\n  T R = clamp_below(sqrt(q * xp",
     "  T yp = sn * dx + cs * dy;\n  T R = clamp_below(sqrt(q * xp"),
    ("sub-pixel offset", "double x = (j - (nx - 1) / 2.0 + (l + 0.5) / ss - 0.5) * D;",
     "double x = (j - (nx - 1) / 2.0 + (l + 0.5) / ss) * D;"),
    ("sub-pixel index transposed", "double x = (j - (nx - 1) / 2.0 + (l + 0.5) / ss - 0.5) * D;",
     "double x = (j - (nx - 1) / 2.0 + (k + 0.5) / ss - 0.5) * D;"),
    ("binning area factor", "acc * (D * D / (ss * ss))", "acc * (1.0 / (ss * ss))"),
    ("correlation instead of convolution", "int ii = i + cy - u, jj = j + cx - v;",
     "int ii = i - cy + u, jj = j - cx + v;"),
    ("PSF not normalised", "(psf[u * kx + v] / sum)", "psf[u * kx + v]"),
    ("likelihood factor", "return -0.5 * chi2;", "return -chi2;"),
    ("residual not whitened", "T r = (s.data[p] - m[p]) / s.sigma[p];", "T r = (s.data[p] - m[p]);"),
    ("truncated normal mass dropped", " - std::log(mass);", ";"),
    ("log-normal Jacobian dropped", "lp = lp - 0.5 * z * z - lx - (std::log(b) + ls2p);",
     "lp = lp - 0.5 * z * z - (std::log(b) + ls2p);"),
    ("uniform density", "lp = lp - std::log(s.prior_hi[k] - s.prior_lo[k]);", "lp = lp;"),
    ("product rule term dropped", "r.d[i] = a.d[i] * b.v + a.v * b.d[i];", "r.d[i] = a.d[i] * b.v;"),
    ("quotient rule sign", "r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);",
     "r.d[i] = (a.d[i] * b.v + a.v * b.d[i]) / (b.v * b.v);"),
    ("atan2 derivative sign", "r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / den;",
     "r.d[i] = (y.v * x.d[i] - x.v * y.d[i]) / den;"),
    ("cos derivative sign", "return chain(a, std::cos(a.v), -std::sin(a.v));",
     "return chain(a, std::cos(a.v), std::sin(a.v));"),
    ("support: gamma bound", "if (!(val(th[1]) > 1.0 && val(th[1]) < 3.0)) return false;",
     "if (!(val(th[1]) > 1.0)) return false;"),
    ("series stops early", "constexpr double SERIES_TOL = 1e-17;", "constexpr double SERIES_TOL = 1e-3;"),
    ("EPL prefactor", "T pref = 2.0 * b / (1.0 + q) * pow(b / R, t - 1.0);",
     "T pref = b / (1.0 + q) * pow(b / R, t - 1.0);"),
    ("EPL slope offset", "T t = p[1] - 1.0;", "T t = p[1] - 2.0;"),
    ("EPL centre sign", "  T dx = x - p[4], dy = y - p[5];\n  T xp = cs * dx + sn * dy;\n  T yp = -sn * dx + cs * dy;\n  T R = clamp_below(sqrt(q * q",
     "  T dx = x + p[4], dy = y - p[5];\n  T xp = cs * dx + sn * dy;\n  T yp = -sn * dx + cs * dy;\n  T R = clamp_below(sqrt(q * q"),
    ("Sersic centre swapped", "  T dx = x - p[4], dy = y - p[5];\n  T xp = cs * dx + sn * dy;\n  T yp = -sn * dx + cs * dy;\n  T R = clamp_below(sqrt(q * xp",
     "  T dx = x - p[5], dy = y - p[4];\n  T xp = cs * dx + sn * dy;\n  T yp = -sn * dx + cs * dy;\n  T R = clamp_below(sqrt(q * xp"),
    ("grid rows not centred", "double y = (i - (ny - 1) / 2.0 + (k + 0.5) / ss - 0.5) * D;",
     "double y = (i - ny / 2.0 + (k + 0.5) / ss - 0.5) * D;"),
    ("PSF centre", "const int cy = (ky - 1) / 2, cx = (kx - 1) / 2;",
     "const int cy = (ky + 1) / 2, cx = (kx - 1) / 2;"),
    ("normal prior quadratic", "lp = lp - 0.5 * z * z - (std::log(b) + ls2p);\n",
     "lp = lp - z * z - (std::log(b) + ls2p);\n"),
    ("sqrt derivative", "return chain(a, s, 0.5 / s);", "return chain(a, s, 1.0 / s);"),
    ("log derivative", "return chain(a, std::log(a.v), 1.0 / a.v);",
     "return chain(a, std::log(a.v), a.v);"),
]

# (module, name, original text, mutated text, pin files) for the Python parts
PY_PINS = {"infer": ["tests/test_oracle_infer.py"], "backward": ["tests/test_oracle_backward.py"],
           "mlp": ["tests/test_oracle_mlp.py"]}
PY_MUTANTS = [
    ("infer", "interval log-det width", "logj += math.log(w) - np.abs(x)", "logj += -np.abs(x)"),
    ("infer", "exp log-det", "th[:, k] = np.exp(x)\n                logj += x",
     "th[:, k] = np.exp(x)\n                logj += 2.0 * x"),
    ("infer", "disc log-det term", " + np.log(_tanh_over(rho))", ""),
    ("infer", "interval Jacobian", "* s * (1.0 - s)", "* s"),
    ("infer", "disc Jacobian outer term", "(g if a == b else 0.0) + gp_over * v[:, a] * v[:, b]",
     "(g if a == b else 0.0)"),
    ("infer", "interval log-det gradient", "G[:, k] = 1.0 - 2.0 / (1.0 + np.exp(-x))",
     "G[:, k] = 1.0 - 1.0 / (1.0 + np.exp(-x))"),
    ("infer", "unconstrained gradient drops the log-det",
     'gu = np.einsum("bij,bi->bj", J, g) + bij.grad_logj(u)', 'gu = np.einsum("bij,bi->bj", J, g)'),
    ("infer", "disc inverse radius", "rho = np.arctanh(r / R)", "rho = np.arctanh(r)"),
    ("infer", "SplitMix64 shift", "z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9)",
     "z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9)"),
    ("infer", "uniform grid offset", "return ((z >> 40) + 0.5)", "return ((z >> 40) + 1.0)"),
    ("infer", "drift without the mass", "u = u + eps * inv_mass * p", "u = u + eps * p"),
    ("infer", "kinetic energy factor", "H0 = -lp + 0.5 * np.sum(inv_mass * p0 * p0, axis=1)",
     "H0 = -lp + np.sum(inv_mass * p0 * p0, axis=1)"),
    ("infer", "momentum scale", "p0 = z / np.sqrt(inv_mass)", "p0 = z * np.sqrt(inv_mass)"),
    ("infer", "acceptance sign", "dH = H0 - H1", "dH = H1 - H0"),
    ("infer", "burn-in fraction", "0.9 * n", "0.5 * n"),
    ("infer", "Adam bias correction", "mh = m / (1 - b1 ** t)\n        vh",
     "mh = m\n        vh"),
    ("infer", "AdaBelief belief term", "d = g - m", "d = g"),
    ("infer", "SVI L-gradient diagonal", "g_L = np.tril(g_L) - np.diag(w.mean() / np.diag(L))",
     "g_L = np.tril(g_L)"),
    ("infer", "SVI score transposed", "a = np.linalg.solve(L.T, z.T).T", "a = np.linalg.solve(L, z.T).T"),
    ("infer", "pathwise mu-gradient sign", "g_mu = -g.sum(0) / n", "g_mu = g.sum(0) / n"),
    ("infer", "pathwise entropy term", "g_L = -np.tril(g.T @ z / n) - np.diag(1.0 / np.diag(L))",
     "g_L = -np.tril(g.T @ z / n)"),
    ("infer", "R-hat between-chain variance",
     "B = N / (M - 1) * ((cm - cm.mean(axis=0)) ** 2).sum(axis=0)",
     "B = 1.0 / (M - 1) * ((cm - cm.mean(axis=0)) ** 2).sum(axis=0)"),
    ("infer", "ESS lag-0 term", "tau = -1.0 + 2.0 * tau_sum", "tau = 2.0 * tau_sum"),
    ("backward", "normal equations weights", "w = (1.0 / system.sigma ** 2).ravel()",
     "w = (1.0 / system.sigma).ravel()"),
    ("backward", "intensity index", "return [8 + 7 * c + 6 for c", "return [8 + 7 * c + 5 for c"),
    ("mlp", "BF16 rounding ties", "(b + 0x7FFF + ((b >> 16) & 1))", "(b + 0x8000)"),
    ("mlp", "SiLU derivative", "sps.append(bf16r(s * (1 + z * (1 - s))))",
     "sps.append(bf16r(s * (1 + z * s)))"),
    ("mlp", "weight gradient input", 'g[f"W{l}"] = bf16(dz).T @ cache[l - 1]',
     'g[f"W{l}"] = bf16(dz).T @ cache[l]'),
    ("mlp", "second series coefficient", "c2 = c1 * (2 + t) / (6 - t)", "c2 = c1 * (2 + t) / (4 - t)"),
    ("mlp", "tail factor power", "return base_F(X) + z ** 3 *", "return base_F(X) + z ** 2 *"),
]

# the pins import the oracle, whose loader builds liboracle.so; the subprocess
# points that build step at the mutant library instead
RUNNER = ("import sys; sys.path[:0] = [{root!r}, {tests!r}]; import oracle.build as b; "
          "b.build = lambda force=False: {lib!r}; import pytest; "
          "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', *{pins!r}]))")

PY_RUNNER = ("import sys, types; sys.path[:0] = [{root!r}, {tests!r}]; import oracle; "
             "path = {path!r}; src = open(path).read(); "
             "m = types.ModuleType('oracle.' + {mod!r}); m.__file__ = path; "
             "m.__package__ = 'oracle'; sys.modules['oracle.' + {mod!r}] = m; "
             "setattr(oracle, {mod!r}, m); "
             "exec(compile(src.replace({old!r}, {new!r}), path, 'exec'), m.__dict__); "
             "import pytest; "
             "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', *{pins!r}]))")


def _pin_python(mod: str, old: str, new: str):
    code = PY_RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"),
                            path=os.path.join(ROOT, "oracle", mod + ".py"), mod=mod, old=old,
                            new=new, pins=PY_PINS[mod])
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-3000:]


def _build_and_pin(tag: str, text: str):
    src = os.path.join(OUT, f"{tag}.cpp")
    lib = os.path.join(OUT, f"lib{tag}.so")
    with open(src, "w") as f:
        f.write(text)
    cc = subprocess.run(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-w",
                         "-o", lib, src], capture_output=True, text=True)
    if cc.returncode != 0:
        return "compile", cc.stderr[-2000:]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib, pins=PINS)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-3000:]


@pytest.fixture(scope="module")
def results():
    src = open(SRC).read()
    jobs = {"original": src}
    for k, (name, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, name
        jobs[f"m{k:02d}"] = src.replace(old, new)
    os.makedirs(OUT, exist_ok=True)
    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {tag: ex.submit(_build_and_pin, tag, text) for tag, text in jobs.items()}
        futs["py-original"] = ex.submit(_pin_python, "infer", "", "")
        for mod in ("backward", "mlp"):
            futs[f"py-original-{mod}"] = ex.submit(_pin_python, mod, "", "")
        for k, (mod, name, old, new) in enumerate(PY_MUTANTS):
            assert open(os.path.join(ROOT, "oracle", mod + ".py")).read().count(old) == 1, name
            futs[f"p{k:02d}"] = ex.submit(_pin_python, mod, old, new)
        return {tag: f.result() for tag, f in futs.items()}


def test_unmodified_oracle_passes_the_pins(results):
    rc, out = results["original"]
    assert rc == 0, out


@pytest.mark.parametrize("k", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(results, k):
    rc, out = results[f"m{k:02d}"]
    assert rc == 1, (MUTANTS[k][0], rc, out)


def test_unmodified_python_oracle_passes_the_pins(results):
    for tag in ("py-original", "py-original-backward", "py-original-mlp"):
        rc, out = results[tag]
        assert rc == 0, (tag, out)


@pytest.mark.parametrize("k", range(len(PY_MUTANTS)), ids=[m[1] for m in PY_MUTANTS])
def test_planted_mistake_in_python_fails_a_pin(results, k):
    rc, out = results[f"p{k:02d}"]
    assert rc == 1, (PY_MUTANTS[k][1], rc, out)
