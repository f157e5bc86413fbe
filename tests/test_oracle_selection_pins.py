"""Pins of the oracle's stencil selection (Sec. 2.5-2.6: eqs. 18-23, Alg. 1 and Alg. 2) and of its
time-step rule, by decisions that flip at thresholds derived here in closed form.

Every case feeds chosen smoothness indicators to the oracle's selection (oracle.select, the
function its reconstruction calls) and checks the cut-off decision just below and just above the
point where chi_1 = C_T, solved by hand from the paper's definitions:

  CTENO (Alg. 1)    gamma_s = lambda_s / (SI_s + eps)^6           (lambda_s of eq. 18: reading R22)
  CTENOZ (Alg. 2)   tau = (sum_{s>=2} |SI_s - SI_1| / (s_t - 1))^6,  gamma_s = lambda_s (1 + tau/(SI_s + eps))
  CTENOZ, reading ctenoz_form = 1 (WENO-Z arrangement): tau unpowered, gamma_s = lambda_s (1 + (tau/(SI_s + eps))^6)
  chi_s = gamma_s / sum_t gamma_t (eq. 22);  delta_s = 0 iff chi_s < C_T (eq. 23)

A wrong exponent, a wrong denominator of tau, a dropped "1 +", a scaled cut-off or a wrong linear
coefficient moves the flip point by far more than the 1e-3 margin the cases use. The time step
(a reading: the paper names only its Courant number) is pinned by the closed-form step of uniform
flow on unjittered meshes whose cells are all congruent.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, select

MARGIN = 1e-3


def _lams(lambda1p, st):
    lam1 = 1.0 - 1.0 / lambda1p
    return lam1, (1.0 - lam1) / (st - 1)


# --------------------------------------------------------------------------------------------
# CTENO (Alg. 1)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("st", [2, 3, 4, 5])
@pytest.mark.parametrize("lambda1p,C_T", [(1e15, 1e-6), (1e4, 1e-6), (1e15, 1e-5), (1e7, 1e-7)])
def test_cteno_central_cutoff_at_closed_form_ratio(st, lambda1p, C_T):
    """Directional indicators all S, central x. chi_1 < C_T  <=>  lam1 (1 - C_T) x^-6 <
    C_T (s_t - 1) lambda_s S^-6, and (s_t - 1) lambda_s = 1/lambda_1' (eq. 18), so the central
    stencil is dropped exactly when (x/S)^6 > (lambda_1' - 1)(1 - C_T)/C_T, for any s_t."""
    r = ((lambda1p - 1.0) * (1.0 - C_T) / C_T) ** (1.0 / 6.0)
    for S in (1e-6, 0.37, 42.0):
        for side, central_kept in ((1 - MARGIN, True), (1 + MARGIN, False)):
            SI = np.array([S * r * side] + [S] * (st - 1))
            bits, chi = select(SI, scheme=0, C_T=C_T, lambda1p=lambda1p, eps=0.0)
            assert bool(bits & 1) == central_kept, (S, side, chi[0] / C_T)
            # the directional stencils all share chi_s = (1 - chi_1)/(s_t - 1) >= C_T
            assert bits >> 1 == (1 << (st - 1)) - 1
            assert abs(chi.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("st", [2, 3, 4])
def test_cteno_cutoff_without_linear_coefficients(st):
    """lam_gamma = 0 (eq. 19 exactly as printed): chi_1 < C_T  <=>  (x/S)^6 > (1 - C_T)/(C_T (s_t-1))."""
    C_T = 1e-6
    r = ((1.0 - C_T) / (C_T * (st - 1))) ** (1.0 / 6.0)
    for side, kept in ((1 - MARGIN, True), (1 + MARGIN, False)):
        bits, _ = select([r * side] + [1.0] * (st - 1), scheme=0, lam_gamma=0, C_T=C_T, eps=0.0)
        assert bool(bits & 1) == kept


def test_cteno_directional_cutoff():
    """Central indicator x, directional S and y (s_t = 3). Directional stencil 3 is cut when
    lambda_s y^-6 (1 - C_T) < C_T (lambda_1 x^-6 + lambda_s S^-6), i.e. for y above
    y* = [C_T (lambda_1 x^-6 / lambda_s + S^-6) / (1 - C_T)]^(-1/6); the other two are kept."""
    C_T, lambda1p = 1e-6, 1e15
    lam1, lams = _lams(lambda1p, 3)
    for x, S in ((1e3, 1.0), (40.0, 0.01)):
        ystar = (C_T * (lam1 * x ** -6 / lams + S ** -6) / (1.0 - C_T)) ** (-1.0 / 6.0)
        for side, kept in ((1 - MARGIN, True), (1 + MARGIN, False)):
            bits, _ = select([x, S, ystar * side], scheme=0, C_T=C_T, lambda1p=lambda1p, eps=0.0)
            assert bool(bits & 4) == kept, (x, S, side)
            assert bits & 2
    # a smooth central stencil (x < S r*) is the only one kept when all directional are rougher
    bits, chi = select([1.0, 5.0, 6.0], scheme=0)
    assert bits == 1 and chi[0] > 1 - 1e-12


def test_cteno_epsilon_enters_as_an_offset():
    """gamma_s = (SI_s + eps)^-6: with every SI = 0 the decisions are those of equal indicators,
    chi_s = lambda_s; with S = 0 and x = (r* - 1) eps (1 -+ margin) the ratio (x + eps)/eps sits at
    the closed-form cut-off r* = ((lambda_1' - 1)(1 - C_T)/C_T)^(1/6)."""
    eps, C_T, lambda1p = 1e-24, 1e-6, 1e15
    bits, chi = select([0.0, 0.0, 0.0], scheme=0, eps=eps)
    lam1, lams = _lams(lambda1p, 3)
    assert np.allclose(chi, [lam1, lams, lams], rtol=1e-14, atol=0) and bits == 1
    r = ((lambda1p - 1.0) * (1.0 - C_T) / C_T) ** (1.0 / 6.0)
    for side, kept in ((1 - MARGIN, True), (1 + MARGIN, False)):
        x = (r * side - 1.0) * eps
        bits, _ = select([x, 0.0, 0.0], scheme=0, eps=eps)
        assert bool(bits & 1) == kept


# --------------------------------------------------------------------------------------------
# Equal indicators: chi_s is the linear coefficient of eq. 18 (both schemes)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,form", [(0, 0), (1, 0), (1, 1)], ids=["CTENO", "CTENOZ", "CTENOZ-wenoz"])
@pytest.mark.parametrize("st", [2, 3, 4, 5])
def test_equal_indicators_give_linear_coefficients(scheme, form, st):
    """All SI equal (tau = 0 for CTENOZ, so gamma_s = lambda_s (1 + 0)): chi_s = lambda_s exactly,
    lambda_1 = 1 - 1/lambda_1' and lambda_s = (1 - lambda_1)/(s_t - 1) (eq. 18). At lambda_1' = 1e15
    only the central stencil survives C_T = 1e-6; at lambda_1' = 2 every stencil does; without the
    linear coefficients chi_s = 1/s_t."""
    for lambda1p in (1e15, 1e4, 2.0):
        lam1, lams = _lams(lambda1p, st)
        bits, chi = select([0.25] * st, scheme=scheme, ctenoz_form=form, lambda1p=lambda1p)
        assert np.allclose(chi, [lam1] + [lams] * (st - 1), rtol=1e-13, atol=0), (lambda1p, chi)
        expect = 1 | (((1 << (st - 1)) - 1) << 1 if lams >= 1e-6 else 0)
        assert bits == expect
    bits, chi = select([0.25] * st, scheme=scheme, ctenoz_form=form, lam_gamma=0)
    assert np.allclose(chi, 1.0 / st, rtol=1e-14) and bits == (1 << st) - 1


@pytest.mark.parametrize("scheme,form", [(0, 0), (1, 0), (1, 1), (2, 0), (3, 0)],
                         ids=["CTENO", "CTENOZ", "CTENOZ-wenoz", "CWENO", "TENO"])
def test_only_the_central_stencil_admissible(scheme, form):
    """The degenerate case s_t = 1 (no admissible directional stencil): eq. 22 normalises a single
    weight, so chi_1 = 1 whatever the indicator, and the central stencil is kept by every scheme
    (eq. 23 with C_T < 1); nothing divides by s_t - 1."""
    for si in (0.0, 1e-30, 0.3, 7.0e5):
        for lambda1p in (1e15, 1e4, 2.0):
            bits, chi = select([si], scheme=scheme, ctenoz_form=form, lambda1p=lambda1p)
            assert bits == 1 and np.array_equal(chi, [1.0]), (si, lambda1p, bits, chi)


# --------------------------------------------------------------------------------------------
# CTENOZ (Alg. 2)
# --------------------------------------------------------------------------------------------
def _ctenoz_flip(x, st, C_T, lambda1p, eps, form):
    """Indicators SI = [x, S, x, ..., x] (one directional stencil S, the other s_t - 2 equal to the
    central x). Then sum_{s>=2} |SI_s - SI_1| = x - S and
      printed form:  tau = ((x - S)/(s_t - 1))^6,   gamma = lambda (1 + tau/(SI + eps));
      WENO-Z form:   tau = (x - S)/(s_t - 1),       gamma = lambda (1 + (tau/(SI + eps))^6).
    With g = the bracket at SI = x and h = the bracket at SI = S, chi_1 < C_T reads
      lambda_1 g (1 - C_T) < C_T lambda_s (h + (s_t - 2) g)   <=>   h > H,
      H = lambda_1 g (1 - C_T) / (C_T lambda_s) - (s_t - 2) g,
    i.e. S + eps < tau / (H - 1) (printed) or tau / (H - 1)^(1/6) (WENO-Z). tau and g depend on S
    only through x - S; the fixed point converges in a few iterations for S << x."""
    lam1, lams = _lams(lambda1p, st)
    S = 0.0
    for _ in range(60):
        if form == 0:
            tau = ((x - S) / (st - 1)) ** 6
            g = 1.0 + tau / (x + eps)
            H = lam1 * g * (1.0 - C_T) / (C_T * lams) - (st - 2) * g
            S_new = tau / (H - 1.0) - eps
        else:
            tau = (x - S) / (st - 1)
            g = 1.0 + (tau / (x + eps)) ** 6
            H = lam1 * g * (1.0 - C_T) / (C_T * lams) - (st - 2) * g
            S_new = tau / (H - 1.0) ** (1.0 / 6.0) - eps
        if S_new == S:
            break
        S = S_new
    return S


@pytest.mark.parametrize("st", [3, 4, 5])
@pytest.mark.parametrize("x", [0.1, 0.5, 2.0])
@pytest.mark.parametrize("lambda1p,C_T", [(1e15, 1e-6), (1e4, 1e-6), (1e15, 1e-5)])
def test_ctenoz_central_cutoff_at_closed_form_point(st, x, lambda1p, C_T):
    eps = 1e-40
    S = _ctenoz_flip(x, st, C_T, lambda1p, eps, 0)
    assert 0.0 < S < 1e-3 * x
    for side, kept in ((1 - MARGIN, False), (1 + MARGIN, True)):
        SI = np.array([x, S * side] + [x] * (st - 2))
        bits, chi = select(SI, scheme=1, C_T=C_T, lambda1p=lambda1p, eps=eps)
        assert bool(bits & 1) == kept, (st, x, side, chi)
        assert bits & 2          # the smooth directional stencil is always kept
        assert abs(chi.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("st", [3, 4, 5])
@pytest.mark.parametrize("x", [0.1, 1.0, 30.0])
def test_ctenoz_wenoz_form_cutoff_and_scale_invariance(st, x):
    """ctenoz_form = 1 (reading: the WENO-Z arrangement). Flip point as derived above; the
    decision depends only on indicator ratios, so scaling every SI by 1e-6 with eps = 0 leaves
    it unchanged."""
    C_T, lambda1p = 1e-6, 1e15
    S = _ctenoz_flip(x, st, C_T, lambda1p, 0.0, 1)
    assert 0.0 < S < x
    for side, kept in ((1 - MARGIN, False), (1 + MARGIN, True)):
        SI = np.array([x, S * side] + [x] * (st - 2))
        for scale in (1.0, 1e-6):
            bits, _ = select(SI * scale, scheme=1, ctenoz_form=1, eps=0.0)
            assert bool(bits & 1) == kept, (st, x, side, scale)


def test_ctenoz_smooth_data_keeps_the_central_stencil():
    """Indicators that differ at O(h^3) relative level (smooth data): tau is tiny, every bracket
    is 1 + O(tau/SI), chi_s ~ lambda_s, and only the central stencil survives (both forms)."""
    for form in (0, 1):
        bits, chi = select([1e-3, 1.001e-3, 0.999e-3, 1.0005e-3], scheme=1, ctenoz_form=form)
        assert bits == 1 and chi[0] > 1 - 1e-12


# --------------------------------------------------------------------------------------------
# Time step (reading R15: dt = CFL min_i |V_i| / sum_f |A_f| (|u.n_f| + c))
# --------------------------------------------------------------------------------------------
def test_time_step_closed_form_2d():
    """Unjittered n x n triangles of legs h, uniform (rho, u, v, p). Each triangle has a horizontal
    leg (normal +-y), a vertical leg (normal +-x) and a hypotenuse of length h sqrt 2 with normal
    (1, +-1)/sqrt 2, so sum_f |A_f|(|u.n_f| + c) = h (|v| + |u| + max|u +- v| + (2 + sqrt 2) c)
    for the cell that limits the step, and dt = CFL (h^2/2) / that."""
    n, cfl = 8, 0.45
    h = 1.0 / n
    rho, u, v, p = 1.3, 0.3, 0.2, 0.9
    c = math.sqrt(1.4 * p / rho)
    expect = cfl * (h * h / 2) / (h * (abs(v) + abs(u) + abs(u) + abs(v) + (2 + math.sqrt(2)) * c))
    for periodic in (True, False):
        mesh = W.tri_mesh(n, n, periodic=periodic, jitter=0.0, seed=4)
        o = Oracle(mesh, setup=False, cfl=cfl)
        o.set_state(W.uniform_state(mesh, [rho, u, v, p]))
        assert abs(o.dt() - expect) < 1e-14 * expect


def test_time_step_closed_form_3d():
    """Unjittered Kuhn tetrahedra (vertices 0, h e_a, h(e_a+e_b), h(e_a+e_b+e_c)): two faces of area
    h^2/2 with normals e_a and e_c, two of area h^2/sqrt 2 with normals (e_a - e_b)/sqrt 2 and
    (e_b - e_c)/sqrt 2. With u = (w, w, w) the last two have u.n = 0, so
    sum_f |A_f|(|u.n_f| + c) = h^2 (w + (1 + sqrt 2) c) and dt = CFL h / (6 (w + (1 + sqrt 2) c))."""
    n, cfl = 4, 0.3
    h = 1.0 / n
    rho, w, p = 0.8, 0.4, 1.7
    c = math.sqrt(1.4 * p / rho)
    expect = cfl * h / (6.0 * (w + (1.0 + math.sqrt(2.0)) * c))
    mesh = W.tet_mesh(n, periodic=True, jitter=0.0)
    o = Oracle(mesh, setup=False, degree=2, cfl=cfl)
    o.set_state(W.uniform_state(mesh, [rho, w, w, w, p]))
    assert abs(o.dt() - expect) < 1e-14 * expect


# --------------------------------------------------------------------------------------------
# CWENO (Sec. 2.3, weights of eq. 14 with b = 4) and TENO (Sec. 2.4)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("st", [2, 3, 4])
@pytest.mark.parametrize("lambda1p", [2.0, 1e4, 1e15])
def test_cweno_weights_closed_form(st, lambda1p):
    """w~_s = lambda_s / (eps + SI_s)^4 normalised. Equal indicators give w_s = lambda_s; with the
    directional indicators y = x (lambda_s / lambda_1)^(1/4) every w~_s is equal, so w_s = 1/s_t.
    Every stencil contributes (all bits)."""
    lam1, lams = _lams(lambda1p, st)
    bits, w = select([0.3] * st, scheme=2, lambda1p=lambda1p, eps=0.0)
    assert bits == (1 << st) - 1
    assert np.allclose(w, [lam1] + [lams] * (st - 1), rtol=1e-13, atol=0)
    x = 0.7
    y = x * (lams / lam1) ** 0.25
    bits, w = select([x] + [y] * (st - 1), scheme=2, lambda1p=lambda1p, eps=0.0)
    assert np.allclose(w, 1.0 / st, rtol=1e-12), w


@pytest.mark.parametrize("st", [2, 3, 4])
def test_teno_cutoff_has_no_linear_coefficients(st):
    """TENO (eqs. 19-23) has no linear coefficients: chi_1 < C_T exactly when
    (x/S)^6 > (1 - C_T)/(C_T (s_t - 1)), whatever lam_gamma says."""
    C_T = 1e-6
    r = ((1.0 - C_T) / (C_T * (st - 1))) ** (1.0 / 6.0)
    for lam_gamma in (0, 1):
        for side, kept in ((1 - MARGIN, True), (1 + MARGIN, False)):
            bits, _ = select([r * side] + [1.0] * (st - 1), scheme=3, lam_gamma=lam_gamma, C_T=C_T, eps=0.0)
            assert bool(bits & 1) == kept


def _poly_field(mesh, degree, rng):
    from tests import exact as X
    V = W.unwrapped_cell_vertices(mesh)
    polys = []
    for v in range(mesh.dim + 2):
        p = X.random_poly(mesh.dim, degree, rng, 0.2)
        p[(0,) * mesh.dim] = 2.0 + v
        polys.append(p)
    U = np.array([[X.poly_cell_average(p, V[c]) for c in range(mesh.ncells)] for p in polys])
    return polys, U


@pytest.mark.parametrize("dim,degree,n", [(2, 2, 8), (2, 3, 10), (3, 2, 5)])
def test_teno_central_polynomial_is_the_least_squares_fit(dim, degree, n):
    """TENO keeps the central stencil's own least-squares polynomial (Sec. 2.4), CTENO the CWENO
    split p_1 = (p_opt - sum lambda_s p_s)/lambda_1 (eq. 17). At lambda_1' = 2 and C_T = 0 (central
    always kept) TENO reproduces a degree-r field exactly; CTENO does not (its p_1 carries the
    directional fits, which are only linear)."""
    from tests import exact as X
    mesh = W.tri_mesh(n, n, periodic=False) if dim == 2 else W.tet_mesh(n, periodic=False)
    polys, U = _poly_field(mesh, degree, np.random.default_rng(41))
    errs = {}
    for scheme in (3, 0):
        o = Oracle(mesh, degree=degree, scheme=scheme, lambda1p=2.0, C_T=0.0, guard=0)
        o.set_state(U)
        o.residual()
        fs = o.face_states()
        fq, _ = o.face_points()
        errs[scheme] = max(np.abs(fs[..., v] - X.poly_eval(polys[v], fq)).max() for v in range(dim + 2))
    assert errs[3] < 1e-11, errs
    assert errs[0] > 1e-4, errs
