"""The synthetic-input priors against the table the paper prints (Eq. sim-dist)."""
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sim_dist.txt")


def _parse_args(kind, text):
    vals = [float(v[2:]) if v.startswith("ln") else float(v) for v in text.split(",")]
    logs = [v.startswith("ln") for v in text.split(",")]
    if kind == "lognormal":
        assert logs[0]
        return synth.LogN(math.log(vals[0]), vals[1])
    if kind == "truncnorm":
        return synth.TN(*vals)
    if kind == "normal":
        return synth.N(*vals)
    if kind == "uniform":
        return synth.U(*vals)
    raise ValueError(kind)


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, kind, sim, pri = line.split()
        rows.append((name, _parse_args(kind, sim), _parse_args(kind, pri)))
    return rows


def _same(a, b):
    return (a.kind == b.kind and math.isclose(a.a, b.a, abs_tol=1e-15) and
            math.isclose(a.b, b.b, abs_tol=1e-15) and
            (a.lo == b.lo or math.isclose(a.lo, b.lo)) and (a.hi == b.hi or math.isclose(a.hi, b.hi)))


def test_paper_prior_columns_match_the_printed_table():
    rows = _golden()
    assert [r[0] for r in rows] == synth.param_names(1, 1)
    sim = synth.paper_prior("simulation").params
    pri = synth.paper_prior("prior").params
    for (name, gs, gp), s, p in zip(rows, sim, pri):
        assert _same(gs, s), name
        assert _same(gp, p), name


def test_benchmark_prior_takes_the_simulation_column_where_unstated():
    """Parameters the benchmark priors leave out (lens centre, lens-light e,
    centre and intensity, source e and intensity) follow the simulation column."""
    rows = dict((r[0], r[1]) for r in _golden())
    spec = synth.config_prior(1, 1)
    names = synth.param_names(1, 1)
    for k in ["epl.x", "epl.y", "shear.gamma1", "shear.gamma2", "light0.e1", "light0.e2",
              "light0.x", "light0.y", "light0.I", "source0.e1", "source0.e2", "source0.I"]:
        assert _same(rows[k], spec.params[names.index(k)]), k


def test_draws_respect_supports():
    spec = synth.config_prior(1, 2)
    th = synth.draw(spec, 500, 9, 1, 2)
    assert th.shape == (500, 29)
    for k, pr in enumerate(spec.params):
        assert np.all(th[:, k] >= pr.lo) and np.all(th[:, k] <= pr.hi)
    assert np.all(np.hypot(th[:, 2], th[:, 3]) < 0.5)
    again = synth.draw(spec, 500, 9, 1, 2)
    np.testing.assert_array_equal(th, again)


def test_psfs_are_normalised_and_centred():
    for k in (synth.moffat_psf(11, 0.262, 1.1), synth.gaussian_core_psf(21, 0.05)):
        assert k.sum() == pytest.approx(1.0, abs=1e-15)
        c = k.shape[0] // 2
        assert np.unravel_index(np.argmax(k), k.shape) == (c, c)
        np.testing.assert_allclose(k, k[::-1, ::-1])
    # Moffat FWHM: half maximum at r = FWHM/2
    D, fwhm = 0.01, 0.2
    k = synth.moffat_psf(41, D, fwhm)
    assert k[20, 30] / k[20, 20] == pytest.approx(0.5, rel=1e-12)
