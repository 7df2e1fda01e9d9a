"""The library's host arithmetic behind every step, without a GPU: the KD
leapfrog factors and the momentum growth of the codec-scale update
(cube_leapfrog_factors, Sections 2.2 and 2.3.3) against 30-digit quadrature
of their definitions and the EdS closed forms, and the step-size bound
(cube_epoch_bound, the host half of cube_next_epoch_limited) against its
closed form in EdS and its defining equation in LCDM."""
import math

import pytest

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 30


@pytest.fixture(scope="module")
def cube():
    from conftest import build_lib
    build_lib()
    import paper_1712_06121_gb300 as c
    return c


def _E(a, om, ol):
    return mpmath.sqrt(om / a ** 3 + (1 - om - ol) / a ** 2 + ol)


def _kick(om, ol, a0, a1):
    return mpmath.quad(lambda a: 1 / (a ** 2 * _E(a, om, ol)), [a0, a1])


def _drift(om, ol, a0, a1):
    return mpmath.quad(lambda a: 1 / (a ** 3 * _E(a, om, ol)), [a0, a1])


def _growth(om, ol, a):
    """g = a^2 E f D with D proportional to E(a) int_0^a dx / (x E)^3 and
    f = d ln D / d ln a taken by numerical differentiation."""
    def lnD(t):
        x = mpmath.exp(t)
        return mpmath.log(_E(x, om, ol) * mpmath.quad(lambda y: 1 / (y * _E(y, om, ol)) ** 3, [0, x]))
    D = mpmath.exp(lnD(mpmath.log(a)))
    f = mpmath.diff(lnD, mpmath.log(a))
    return a ** 2 * _E(a, om, ol) * f * D


@pytest.mark.parametrize("om,ol", [(0.3, 0.7), (0.3, 0.0), (1 - 1e-12, 0.0)])
@pytest.mark.parametrize("a0,a1", [(0.02, 1.0), (0.1, 0.1002), (0.5, 0.9), (1.0, 0.5)])
def test_leapfrog_factors_match_their_integrals(cube, om, ol, a0, a1):
    """Quadrature path (no closed form): within 1e-13 of 30-digit values.
    The near-EdS case checks the quadrature against EdS's closed forms too."""
    k, d, g = cube.cube_leapfrog_factors(om, ol, a0, a1)
    m = [mpmath.mpf(x) for x in (om, ol, a0, a1)]
    assert k == pytest.approx(float(_kick(*m)), rel=1e-13)
    assert d == pytest.approx(float(_drift(*m)), rel=1e-13)
    assert g == pytest.approx(float(_growth(m[0], m[1], m[3]) / _growth(m[0], m[1], m[2])), rel=1e-12)


@pytest.mark.parametrize("a0,a1", [(0.02, 0.04), (0.3, 1.0)])
def test_leapfrog_factors_eds(cube, a0, a1):
    k, d, g = cube.cube_leapfrog_factors(1.0, 0.0, a0, a1)
    assert k == pytest.approx(2 * (math.sqrt(a1) - math.sqrt(a0)), rel=1e-15)
    assert d == pytest.approx(2 * (1 / math.sqrt(a0) - 1 / math.sqrt(a1)), rel=1e-15)
    assert g == pytest.approx((a1 / a0) ** 1.5, rel=1e-15)                    # D = a, f = 1


def test_zero_interval(cube):
    assert cube.cube_leapfrog_factors(0.3, 0.7, 0.4, 0.4) == (0.0, 0.0, 1.0)


def test_epoch_bound_eds_closed_form(cube):
    """F_max = 0 in EdS: p 2 (a^-1/2 - a_to^-1/2) = cells R gives
    a_to = (a^-1/2 - cells R / (2 p))^-2."""
    a, R, p, cells = 0.1, 4, 3.0, 0.5
    want = (a ** -0.5 - cells * R / (2 * p)) ** -2
    got, why = cube.cube_epoch_bound(1.0, 0.0, R, a, a, 1.0, p, 0.0, drift_cells=cells)
    assert why == 1 and got == pytest.approx(want, rel=1e-13)
    # a_max below that: a_max itself; an expansion limit below both: a e^dlna
    assert cube.cube_epoch_bound(1.0, 0.0, R, a, a, 0.9 * want, p, 0.0, drift_cells=cells) == (0.9 * want, 0)
    got, why = cube.cube_epoch_bound(1.0, 0.0, R, a, a, 1.0, p, 0.0, drift_cells=cells, max_dlna=0.01)
    assert why == 2 and got == pytest.approx(a * math.exp(0.01), rel=1e-15)
    # nothing moves: no drift limit
    assert cube.cube_epoch_bound(1.0, 0.0, R, a, a, 1.0, 0.0, 0.0) == (1.0, 0)


@pytest.mark.parametrize("a,a_p", [(0.2, 0.2), (0.5, 0.49)])
def test_epoch_bound_with_force_solves_its_equation(cube, a, a_p):
    """LCDM with F_max > 0: the returned a_to makes
    (p + F int_{a_p}^{(a + a_to)/2} da/(a^2 E)) int_a^{a_to} da/(a^3 E)
    equal to cells R (the left side grows with a_to), and the force shortens
    the step."""
    om, ol, R, p, f, cells = 0.3, 0.7, 4, 2.0, 40.0, 0.25
    got, why = cube.cube_epoch_bound(om, ol, R, a, a_p, 1.0, p, f, drift_cells=cells)
    m = [mpmath.mpf(x) for x in (om, ol, a, a_p, got)]
    lhs = (p + f * _kick(m[0], m[1], m[3], (m[2] + m[4]) / 2)) * _drift(m[0], m[1], m[2], m[4])
    assert why == 1 and float(lhs) == pytest.approx(cells * R, rel=1e-12)
    no_force, _ = cube.cube_epoch_bound(om, ol, R, a, a_p, 1.0, p, 0.0, drift_cells=cells)
    assert a < got < no_force


@pytest.mark.parametrize("kw", [dict(drift_cells=0.0), dict(drift_cells=1.5), dict(max_dlna=-0.1)])
def test_epoch_bound_rejects_bad_limits(cube, kw):
    with pytest.raises(cube.CubeError) as e:
        cube.cube_epoch_bound(0.3, 0.7, 4, 0.1, 0.1, 0.2, 1.0, 0.0, **kw)
    assert e.value.status == cube.CUBE_E_ARG


@pytest.mark.parametrize("args", [(0.3, 0.7, 4, 0.1, 0.1, 0.1, 1.0, 0.0),          # a_max = a
                                  (0.3, 0.7, 4, 0.1, 0.2, 0.3, 1.0, 0.0),          # a_p > a
                                  (0.0, 0.7, 4, 0.1, 0.1, 0.3, 1.0, 0.0),          # omega_m = 0
                                  (0.3, 0.7, 0, 0.1, 0.1, 0.3, 1.0, 0.0),          # ratio 0
                                  (0.3, 0.7, 4, 0.1, 0.1, 0.3, -1.0, 0.0),         # p_max < 0
                                  (0.3, 0.7, 4, 0.1, 0.1, 0.3, 1e300, 0.0)])       # no positive step
def test_epoch_bound_argument_errors(cube, args):
    with pytest.raises(cube.CubeError) as e:
        cube.cube_epoch_bound(*args)
    assert e.value.status == cube.CUBE_E_ARG
    assert cube.cube_last_error()


def test_leapfrog_factors_argument_errors(cube):
    for args in ((0.0, 0.7, 0.1, 0.2), (0.3, -0.1, 0.1, 0.2), (0.3, 0.7, 0.0, 0.2), (0.3, 0.7, 0.1, -1.0)):
        with pytest.raises(cube.CubeError) as e:
            cube.cube_leapfrog_factors(*args)
        assert e.value.status == cube.CUBE_E_ARG
