"""Pins of the CPU oracle against mathematics other than itself.

Each test ties one part of the oracle to something it does not compute
itself: a printed closed form, a textbook rule, a hand-worked example, an
identity of the Legendre family, an exactness property of the quadrature, an
invariance of the method, or an independent derivative (complex step, finite
differences, PyTorch autograd).  A plausible mistake in the oracle (a dropped
term, a sign, a swapped xi/eta, a transposed operand) fails at least one.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import fv_inputs as fi
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature
def _load_gll_golden():
    rows = {}
    for line in open(os.path.join(GOLDEN, "gll_textbook.txt")):
        if line.startswith("#") or not line.strip():
            continue
        Q, x, w = line.split()
        rows.setdefault(int(Q), []).append((float(x), float(w)))
    return rows


def test_gll_matches_textbook_closed_forms():
    for Q, nw in _load_gll_golden().items():
        x, w = oracle.gll(Q)
        np.testing.assert_allclose(x, [a for a, _ in nw], rtol=0, atol=1e-15)
        np.testing.assert_allclose(w, [b for _, b in nw], rtol=1e-14, atol=0)


@pytest.mark.parametrize("Q", [2, 3, 4, 5, 8, 10, 13, 20])
def test_gll_exactness_and_first_failure(Q):
    x, w = oracle.gll(Q)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * Q - 2):                       # exact through degree 2Q-3
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13, k
    # degree 2Q-2: Lobatto error term (Abramowitz & Stegun 25.4.32)
    #   int f - sum w f = -Q (Q-1)^3 2^(2Q-1) ((Q-2)!)^4 / ((2Q-1) ((2Q-2)!)^3) f^(2Q-2)
    k = 2 * Q - 2
    err = (2.0 / (k + 1)) - np.dot(w, x ** k)
    c = -Q * (Q - 1) ** 3 * 2.0 ** (2 * Q - 1) * math.factorial(Q - 2) ** 4 / (
        (2 * Q - 1) * math.factorial(2 * Q - 2) ** 3) * math.factorial(2 * Q - 2)
    assert err < 0                                      # the rule over-integrates x^(2Q-2)
    assert abs(err - c) < 1e-12 * max(1.0, abs(c)), (err, c)


# ---------------------------------------------------------------- Legendre / test functions
def test_legendre_against_numpy():
    s = np.linspace(-1, 1, 41)
    for n in range(0, 12):
        P, dP = oracle.legendre(n, s)
        coef = np.zeros(n + 1); coef[n] = 1.0
        np.testing.assert_allclose(P, npleg.legval(s, coef), atol=1e-13)
        np.testing.assert_allclose(dP, npleg.legval(s, npleg.legder(coef)), atol=1e-11)


def test_test_functions_identities():
    s = np.linspace(-1, 1, 33)
    xg, wg = npleg.leggauss(40)
    for n in range(1, 12):
        v, dv = oracle.test_fn(n, np.array([-1.0, 1.0]))
        assert np.all(np.abs(v) < 1e-14)                  # v_n vanishes on the element boundary
        v, dv = oracle.test_fn(n, s)
        P, _ = oracle.legendre(n, s)
        np.testing.assert_allclose(dv, (2 * n + 1) * P, atol=1e-11)   # v_n' = (2n+1) P_n
        vg, _ = oracle.test_fn(n, xg)
        integral = float(np.dot(wg, vg))
        assert abs(integral - (-2.0 if n == 1 else 0.0)) < 1e-13


# ---------------------------------------------------------------- bilinear map
def test_bilinear_hand_worked_example():
    kv = {}
    for line in open(os.path.join(GOLDEN, "bilinear_worked_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *vals = line.split()
        kv[k] = [float(v) for v in vals]
    out = oracle.map_points(kv["vx"], kv["vy"], kv["xi"], kv["eta"])[0]
    for i, key in enumerate(["x", "y", "x_xi", "x_eta", "y_xi", "y_eta", "D"]):
        assert abs(out[i] - kv[key][0]) < 1e-15, key


def test_jacobian_against_finite_differences_and_area():
    prob = fi.skewed_disc()
    h = 1e-6
    rng = fi.SplitMix64(7, 9)
    for e in range(0, prob.mesh.n_elements, 37):
        c = prob.mesh.cells[e]
        vx, vy = prob.mesh.vertices[c, 0], prob.mesh.vertices[c, 1]
        xi, eta = 2 * rng.uniform() - 1, 2 * rng.uniform() - 1
        o = oracle.map_points(vx, vy, [xi, xi + h, xi - h, xi, xi], [eta, eta, eta, eta + h, eta - h])
        assert abs((o[1, 0] - o[2, 0]) / (2 * h) - o[0, 2]) < 1e-8
        assert abs((o[3, 0] - o[4, 0]) / (2 * h) - o[0, 3]) < 1e-8
        assert abs((o[1, 1] - o[2, 1]) / (2 * h) - o[0, 4]) < 1e-8
        assert abs((o[3, 1] - o[4, 1]) / (2 * h) - o[0, 5]) < 1e-8
        # corners land on the vertices
        oc = oracle.map_points(vx, vy, [-1, 1, 1, -1], [-1, -1, 1, 1])
        np.testing.assert_allclose(oc[:, 0], vx, atol=1e-15)
        np.testing.assert_allclose(oc[:, 1], vy, atol=1e-15)
    # sum_q w_q D_q equals the shoelace area exactly (D is bilinear)
    for Q in (2, 3, 5):
        geo = oracle.geometry(prob.mesh, Q)
        x, w = oracle.gll(Q)
        W = np.outer(w, w).ravel()
        v = prob.mesh.vertices[prob.mesh.cells]
        shoelace = 0.5 * np.sum(v[..., 0] * np.roll(v[..., 1], -1, 1) - np.roll(v[..., 0], -1, 1) * v[..., 1], 1)
        np.testing.assert_allclose((geo[..., 6] * W).sum(1), shoelace, rtol=1e-13)


def _skewed_mesh(n=3, seed=5):
    base = fi.rect_grid(n, n)
    return fi.jitter_nodes(base, ~fi.boundary_nodes_of(base), 0.25, seed=seed)


def test_physical_gradients_against_linear_solve():
    """G_x / (w D) and G_y / (w D) must be grad(v) obtained by solving the
    2x2 Jacobian system at every node (an independent route to the true
    inverse Jacobian; the printed inverse in App. A.1 swaps xi/eta)."""
    Q, T = 4, 3
    mesh = _skewed_mesh()
    prob = fi.Problem("skew", mesh, Q, T, [2, 4, 1], np.zeros(17), lambda x, y: 0 * x, lambda x, y: 0 * x,
                      np.zeros((0, 2)), np.zeros(0))
    Gx, Gy, Gv, F = oracle.Bound(prob, with_boundary=False).tensors()
    geo = oracle.geometry(mesh, Q)
    xs, ws = oracle.gll(Q)
    for e in range(mesh.n_elements):
        for a in range(Q):
            for b in range(Q):
                q = a * Q + b
                x_xi, x_eta, y_xi, y_eta, D = geo[e, q, 2:]
                J = np.array([[x_xi, y_xi], [x_eta, y_eta]])   # rows: d/dxi, d/deta of (x, y)
                for m in range(1, T + 1):
                    for n in range(1, T + 1):
                        cm = np.zeros(m + 2); cm[m + 1] = 1; cm[m - 1] -= 1
                        cn = np.zeros(n + 2); cn[n + 1] = 1; cn[n - 1] -= 1
                        vm, dvm = npleg.legval(xs[a], cm), npleg.legval(xs[a], npleg.legder(cm))
                        vn, dvn = npleg.legval(xs[b], cn), npleg.legval(xs[b], npleg.legder(cn))
                        gx, gy = np.linalg.solve(J, [dvm * vn, vm * dvn])
                        j = (m - 1) * T + (n - 1)
                        wD = ws[a] * ws[b] * D
                        assert abs(Gx[e, j, q] - wD * gx) < 1e-13
                        assert abs(Gy[e, j, q] - wD * gy) < 1e-13
                        assert abs(Gv[e, j, q] - wD * vm * vn) < 1e-13


def test_axis_aligned_reduces_to_algorithm2_scaling():
    """On axis-aligned rectangles G_x = w (D / x_xi) v_xi  (Algorithm 2's J_x = j / j_x, App. A.2)."""
    Q, T = 5, 4
    mesh = fi.rect_grid(3, 2, 0.0, 1.5, 0.0, 0.4)
    prob = fi.Problem("rect", mesh, Q, T, [2, 4, 1], np.zeros(17), lambda x, y: 0 * x, lambda x, y: 0 * x,
                      np.zeros((0, 2)), np.zeros(0))
    Gx, Gy, _, _ = oracle.Bound(prob, with_boundary=False).tensors()
    xs, ws = oracle.gll(Q)
    hx, hy = 1.5 / 3, 0.4 / 2
    j_det, jx, jy = hx * hy / 4, hx / 2, hy / 2
    for m in range(1, T + 1):
        for n in range(1, T + 1):
            vm, dvm = oracle.test_fn(m, xs)
            vn, dvn = oracle.test_fn(n, xs)
            Vx = np.outer(ws * dvm, ws * vn).ravel()          # reference premultiplier (w v_xi)
            Vy = np.outer(ws * vm, ws * dvn).ravel()
            j = (m - 1) * T + (n - 1)
            for e in range(mesh.n_elements):
                np.testing.assert_allclose(Gx[e, j], (j_det / jx) * Vx, atol=1e-14)
                np.testing.assert_allclose(Gy[e, j], (j_det / jy) * Vy, atol=1e-14)


def test_mass_premultiplier_sums_on_parallelograms():
    """sum_q Gv[e,j,q] = (area/4) (int v_m)(int v_n): the element area for j=(1,1), 0 otherwise."""
    Q, T = 6, 4   # Q >= (T+4)/2
    mesh = fi.rect_grid(2, 2)
    v = mesh.vertices.copy()
    v[:, 0] += 0.3 * v[:, 1]          # shear: parallelograms
    mesh = fi.Mesh(v, mesh.cells)
    prob = fi.Problem("para", mesh, Q, T, [2, 4, 1], np.zeros(17), lambda x, y: 0 * x, lambda x, y: 0 * x,
                      np.zeros((0, 2)), np.zeros(0))
    _, _, Gv, _ = oracle.Bound(prob, with_boundary=False).tensors()
    s = Gv.sum(2)
    area = 0.25
    for j in range(T * T):
        expect = area if j == 0 else 0.0
        np.testing.assert_allclose(s[:, j], expect, atol=1e-14)


# ---------------------------------------------------------------- residual
def _with(prob, **kw):
    d = dict(prob.__dict__)
    d.update(kw)
    return fi.Problem(**d)


@pytest.mark.parametrize("T,Q", [(3, 4), (5, 5), (6, 5), (4, 8)])
def test_linear_patch_test_on_skewed_mesh(T, Q):
    """u = alpha x + beta y + gamma, f = 0: every cell residual vanishes (v = 0 on
    the cell boundary), exactly when the rule integrates degree T+1 per variable."""
    mesh = _skewed_mesh(4, seed=11)
    prob = fi.Problem("patch", mesh, Q, T, [2, 4, 1], np.zeros(17), lambda x, y: 0 * x, lambda x, y: 0 * x,
                      np.zeros((0, 2)), np.zeros(0), eps=0.7)
    b = oracle.Bound(prob, with_boundary=False)
    n = mesh.n_elements * Q * Q
    R = b.residuals_given_grad(np.full(n, 1.7), np.full(n, -0.6))
    exact = Q >= (T + 4) / 2
    if exact:
        assert np.max(np.abs(R)) < 1e-13
    else:
        assert np.max(np.abs(R)) > 1e-8   # under-integrated: the patch test must fail


def test_manufactured_solution_residual_vanishes_with_quadrature():
    """With u = the exact solution and f = -Lap u, |R| -> 0 as Q grows."""
    base = fi.tiny_square()
    uex = lambda x, y: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    gx = lambda x, y: 2 * np.pi * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    gy = lambda x, y: 2 * np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    prev = None
    for Q in (4, 5, 6, 8, 10, 20):
        prob = _with(base, quad_order=Q)
        b = oracle.Bound(prob, with_boundary=False)
        X = oracle.quad_points(prob.mesh, Q).reshape(-1, 2)
        R = b.residuals_given_grad(gx(X[:, 0], X[:, 1]), gy(X[:, 0], X[:, 1]))
        Fn = np.max(np.abs(b.tensors()[3]))
        rel = np.max(np.abs(R)) / Fn
        if prev is not None:
            assert rel < prev or rel < 1e-13     # decreasing until the roundoff floor
        prev = rel
    assert prev < 1e-12


def test_loop_variant_equals_tensor_variant():
    prob = _with(fi.skewed_disc(), b=(0.3, -0.2), eps=0.8)
    prob.mesh = prob.mesh.subset(0, 96)
    b = oracle.Bound(prob, with_boundary=False)
    out = b.loss_grad(prob.params, want_grad=False, want_R=True, want_upts=True)
    Gx, Gy, Gv, F = b.tensors()
    up = out["upts"]
    R2 = oracle.contract(Gx, Gy, Gv, F, up[..., 1], up[..., 2], prob.eps, 0.3, -0.2)
    np.testing.assert_allclose(R2, out["R"], rtol=0, atol=1e-14 * np.max(np.abs(out["R"])))


def test_loss_invariant_under_cell_vertex_rotation_and_element_order():
    """Cyclically relabelling each cell's vertices rotates the reference square by
    90 degrees; the tensor-product test space maps to itself up to signs, so
    the loss is unchanged.  So is any permutation of the elements."""
    prob = fi.skewed_disc()
    prob.mesh = prob.mesh.subset(200, 264)
    base = oracle.Bound(prob).loss_value(prob.params)
    for shift in (1, 2, 3):
        cells = np.roll(prob.mesh.cells, shift, axis=1)
        p2 = _with(prob, mesh=fi.Mesh(prob.mesh.vertices, cells))
        np.testing.assert_allclose(oracle.Bound(p2).loss_value(prob.params), base, rtol=1e-13)
    perm = np.array(fi.SplitMix64(3, 5).uniforms(64)).argsort()
    p3 = _with(prob, mesh=fi.Mesh(prob.mesh.vertices, prob.mesh.cells[perm]))
    np.testing.assert_allclose(oracle.Bound(p3).loss_value(prob.params), base, rtol=1e-13)


def test_norm_conventions_ratio():
    """Algorithm 3 (mean over tests) and Eq. (loss) (mean over elements) differ by N_t / N_e."""
    prob = fi.tiny_square()
    Lt = oracle.Bound(prob, norm=0).loss_value(prob.params)[1]
    Le = oracle.Bound(prob, norm=1).loss_value(prob.params)[1]
    assert abs(Le / Lt - prob.test_order ** 2 / prob.mesh.n_elements) < 1e-13


# ---------------------------------------------------------------- MLP and gradients
def test_mlp_gradient_complex_step_and_fd():
    prob = fi.gear_annulus()
    xy = fi.uniform_points(64, 1, 7)
    u, ux, uy = oracle.mlp(prob.widths, prob.params, xy)
    cx, cy = oracle.mlp_cstep_x(prob.widths, prob.params, xy)
    np.testing.assert_allclose(ux, cx, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(uy, cy, rtol=1e-13, atol=1e-15)
    h = 1e-6
    up, _, _ = oracle.mlp(prob.widths, prob.params, xy + [h, 0])
    um, _, _ = oracle.mlp(prob.widths, prob.params, xy - [h, 0])
    np.testing.assert_allclose(ux, (up - um) / (2 * h), atol=1e-8)


def test_mlp_value_independent_numpy():
    """The forward value against a direct numpy evaluation of Eq. (NN)."""
    prob = fi.skewed_disc()
    xy = fi.uniform_points(50, 2, 7)
    u, _, _ = oracle.mlp(prob.widths, prob.params, xy)
    h = xy.T
    off = 0
    ws = prob.widths
    for i in range(len(ws) - 1):
        W = prob.params[off: off + ws[i + 1] * ws[i]].reshape(ws[i + 1], ws[i]); off += ws[i + 1] * ws[i]
        bb = prob.params[off: off + ws[i + 1]]; off += ws[i + 1]
        h = W @ h + bb[:, None]
        if i + 1 < len(ws) - 1:
            h = np.tanh(h)
    np.testing.assert_allclose(u, h[0], rtol=1e-13, atol=1e-15)


def test_full_gradient_complex_step_small_problem():
    """Every parameter and eps, CD2D with boundary and sensor terms, on a tiny problem."""
    mesh = _skewed_mesh(2, seed=2)
    widths = [2, 6, 5, 1]
    params = fi.random_bias_params(widths, 9, 1, gain=1.3)
    u, f = fi.sinsin(2 * math.pi)
    bd = fi.square_boundary_points(5)
    sens = fi.uniform_points(7, 9, 2, 0, 1)
    prob = fi.Problem("tiny", mesh, 5, 4, widths, params, u, f, bd, u(bd[:, 0], bd[:, 1]) + 0.1, eps=0.45,
                      b=(0.3, -0.7), tau=3.0, sensor_xy=sens, sensor_u=u(sens[:, 0], sens[:, 1]), gamma=2.0)
    for norm in (0, 1):
        b = oracle.Bound(prob, norm=norm)
        out = b.loss_grad(params)
        idx = np.arange(len(params))
        cs = b.cstep(params, np.concatenate([idx, [-1]]))
        np.testing.assert_allclose(out["grad"], cs[:-1], rtol=1e-12, atol=1e-14 * np.abs(cs).max())
        assert abs(out["dL_deps"] - cs[-1]) < 1e-12 * abs(cs[-1])


def test_tiny_gradient_complex_step_subset_and_fd():
    prob = fi.tiny_square()
    b = oracle.Bound(prob)
    out = b.loss_grad(prob.params)
    idx = np.arange(0, len(prob.params), 23)
    cs = b.cstep(prob.params, idx, n_threads=4)
    np.testing.assert_allclose(out["grad"][idx], cs, rtol=1e-11, atol=1e-13 * np.abs(cs).max())
    # central finite differences on a few coordinates
    for i in idx[:6]:
        h = 1e-6 * max(1.0, abs(prob.params[i]))
        pp, pm = prob.params.copy(), prob.params.copy()
        pp[i] += h; pm[i] -= h
        fd = (b.loss_value(pp)[0] - b.loss_value(pm)[0]) / (2 * h)
        assert abs(fd - out["grad"][i]) < 1e-6 * max(1.0, abs(out["grad"][i]))


def test_loss_is_quadratic_in_eps():
    """R is affine in eps, so L(eps) is a parabola: three values fix dL/deps and d2L/deps2."""
    prob = fi.inverse_cd2d(8)
    b = oracle.Bound(prob)
    e0 = 0.9
    Ls = [b.loss_value(prob.params, eps=e)[0] for e in (e0 - 0.5, e0, e0 + 0.5)]
    d1 = (Ls[2] - Ls[0]) / 1.0
    out = b.loss_grad(prob.params, eps=e0)
    assert abs(out["dL_deps"] - d1) < 1e-10 * max(1.0, abs(d1))
    L4 = b.loss_value(prob.params, eps=e0 + 1.3)[0]
    c2 = (Ls[2] - 2 * Ls[1] + Ls[0]) / 0.25 / 2
    pred = Ls[1] + d1 * 1.3 + c2 * 1.3 ** 2
    assert abs(L4 - pred) < 1e-10 * abs(L4)


def test_gradient_against_torch_double_backward():
    """The hand-written reverse sweep against PyTorch CPU FP64 autograd
    (grad u by create_graph autograd, then backward) on the tensor form."""
    torch = pytest.importorskip("torch")
    prob = fi.tiny_square()
    prob = _with(prob, b=(0.2, 0.1), eps=0.8, params=fi.random_bias_params(prob.widths, 1, 1))
    b = oracle.Bound(prob)
    out = b.loss_grad(prob.params)
    Gx, Gy, Gv, F = (torch.tensor(a) for a in b.tensors())
    X = torch.tensor(oracle.quad_points(prob.mesh, prob.quad_order).reshape(-1, 2))
    theta = torch.tensor(prob.params, requires_grad=True)
    ws = prob.widths

    def net(xy):
        h, off = xy, 0
        for i in range(len(ws) - 1):
            W = theta[off: off + ws[i + 1] * ws[i]].view(ws[i + 1], ws[i]); off += ws[i + 1] * ws[i]
            bb = theta[off: off + ws[i + 1]]; off += ws[i + 1]
            h = h @ W.T + bb
            if i + 1 < len(ws) - 1:
                h = torch.tanh(h)
        return h[:, 0]

    Xr = X.clone().requires_grad_(True)
    u = net(Xr)
    (g,) = torch.autograd.grad(u.sum(), Xr, create_graph=True)
    ne, nq = Gx.shape[0], Gx.shape[2]
    ux, uy = g[:, 0].view(ne, nq), g[:, 1].view(ne, nq)
    R = prob.eps * (torch.einsum("ejq,eq->ej", Gx, ux) + torch.einsum("ejq,eq->ej", Gy, uy)) \
        + torch.einsum("ejq,eq->ej", Gv, prob.b[0] * ux + prob.b[1] * uy) - F
    Lv = (R ** 2).mean(1).sum()
    ub = net(torch.tensor(prob.bd_xy))
    Lb = ((ub - torch.tensor(prob.bd_g)) ** 2).mean()
    L = Lv + prob.tau * Lb
    L.backward()
    assert abs(L.item() - out["loss"]) < 1e-12 * out["loss"]
    np.testing.assert_allclose(theta.grad.numpy(), out["grad"], rtol=1e-10,
                               atol=1e-12 * np.abs(out["grad"]).max())


def test_adjoint_seeds_are_dL_dgradu():
    """ubar at a node = dLv / d(u_x, u_y) there: perturb one node's u_x in the
    given-gradient residual and difference Lv."""
    prob = _with(fi.tiny_square(), b=(0.4, 0.0), eps=0.6)
    b = oracle.Bound(prob, with_boundary=False)
    out = b.loss_grad(prob.params, want_ubar=True, want_upts=True)
    up = out["upts"].reshape(-1, 3)
    Nt = prob.test_order ** 2
    for node in (0, 7, 131, 399):
        for comp in (0, 1):
            h = 1e-6
            vals = []
            for s in (+1, -1):
                ux, uy = up[:, 1].copy(), up[:, 2].copy()
                (ux if comp == 0 else uy)[node] += s * h
                R = b.residuals_given_grad(ux, uy)
                vals.append((R ** 2).sum() / Nt)
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - out["ubar"].reshape(-1, 2)[node, comp]) < 1e-6 * max(1, abs(fd))


def test_boundary_and_sensor_terms():
    prob = fi.inverse_cd2d(4)
    out = oracle.Bound(prob).loss_grad(prob.params)
    u, _, _ = oracle.mlp(prob.widths, prob.params, prob.bd_xy)
    us, _, _ = oracle.mlp(prob.widths, prob.params, prob.sensor_xy)
    assert abs(out["Lb"] - np.mean((u - prob.bd_g) ** 2)) < 1e-14 * out["Lb"]
    assert abs(out["Ls"] - np.mean((us - prob.sensor_u) ** 2)) < 1e-14 * out["Ls"]
    assert abs(out["loss"] - (out["Lv"] + prob.tau * out["Lb"] + prob.gamma * out["Ls"])) < 1e-13 * out["loss"]


def test_inverse_problem_source_term():
    """f = -eps u'' + b u' for the inverse problem's exact u (hand-derived
    derivatives) against finite differences."""
    u, f, up, upp = fi.inverse_exact(0.3, 0.3, 0.1)
    x = np.linspace(-1, 1, 21)
    h = 1e-4
    np.testing.assert_allclose(up(x, 0), (u(x + h, 0) - u(x - h, 0)) / (2 * h), atol=1e-7)
    np.testing.assert_allclose(upp(x, 0), (u(x + h, 0) - 2 * u(x, 0) + u(x - h, 0)) / h ** 2, atol=1e-5)


# ---------------------------------------------------------------- space-dependent eps (Sec. 4.7.2)
def _two_output_params(widths1, params1, eps0):
    """A two-output network whose second output is the constant eps0: the
    first output's weights are params1's, the eps row is zero, its bias eps0."""
    n_in = widths1[-2]
    head = params1[:len(params1) - (n_in + 1)]
    W_u, b_u = params1[len(params1) - (n_in + 1): len(params1) - 1], params1[-1]
    return np.concatenate([head, W_u, np.zeros(n_in), [b_u, eps0]])


def test_eps_field_reduces_to_constant_eps():
    """A two-output network with a constant second output eps0 gives the loss of
    the scalar-eps problem at eps0, the same gradient on the shared weights, and
    on the eps bias exactly dL/deps of the scalar problem (which is pinned by
    complex step above)."""
    mesh = _skewed_mesh(2, seed=5)
    widths1 = [2, 6, 5, 1]
    params1 = fi.random_bias_params(widths1, 4, 1, gain=1.2)
    u, f = fi.sinsin(2 * math.pi)
    bd = fi.square_boundary_points(5)
    eps0 = 0.65
    prob1 = fi.Problem("tiny", mesh, 5, 4, widths1, params1, u, f, bd, u(bd[:, 0], bd[:, 1]), eps=eps0,
                       b=(0.3, -0.2), tau=2.0)
    widths2 = widths1[:-1] + [2]
    params2 = _two_output_params(widths1, params1, eps0)
    prob2 = fi.Problem("tiny2", mesh, 5, 4, widths2, params2, u, f, bd, u(bd[:, 0], bd[:, 1]), eps=123.0,
                       b=(0.3, -0.2), tau=2.0)
    r1 = oracle.Bound(prob1).loss_grad(params1)
    r2 = oracle.Bound(prob2).loss_grad(params2, want_eps_field=True)
    assert abs(r2["loss"] - r1["loss"]) < 1e-13 * abs(r1["loss"])
    n_in = widths1[-2]
    head = len(params1) - (n_in + 1)
    np.testing.assert_allclose(r2["grad"][:head + n_in], r1["grad"][:head + n_in], rtol=1e-12, atol=1e-15)
    assert abs(r2["grad"][head + 2 * n_in] - r1["grad"][-1]) < 1e-12 * abs(r1["grad"][-1])     # b_u
    assert abs(r2["grad"][-1] - r1["dL_deps"]) < 1e-12 * abs(r1["dL_deps"])                    # b_eps
    assert r2["dL_deps"] == 0.0
    np.testing.assert_allclose(r2["epts"], eps0, rtol=0, atol=1e-15)
    # the eps seeds sum to dL/deps over the whole mesh
    assert abs(r2["ebar"].sum() - r1["dL_deps"]) < 1e-12 * abs(r1["dL_deps"])


def test_eps_field_gradient_complex_step():
    """Every parameter of a two-output network (u, eps(x, y)) on a tiny CD2D
    problem with boundary and sensor terms, against complex-step derivatives
    of the loss (the generic loss code shares nothing with the reverse sweep)."""
    mesh = _skewed_mesh(2, seed=6)
    widths = [2, 5, 6, 2]
    params = fi.random_bias_params(widths, 11, 1, gain=1.1)
    u, f = fi.sinsin(2 * math.pi)
    bd = fi.square_boundary_points(4)
    sens = fi.uniform_points(5, 12, 2, 0, 1)
    prob = fi.Problem("tiny-eps-field", mesh, 5, 4, widths, params, u, f, bd, u(bd[:, 0], bd[:, 1]), eps=7.0,
                      b=(0.5, 0.25), tau=1.5, sensor_xy=sens, sensor_u=u(sens[:, 0], sens[:, 1]) + 0.05, gamma=3.0)
    b = oracle.Bound(prob)
    out = b.loss_grad(params)
    cs = b.cstep(params, np.arange(len(params)))
    np.testing.assert_allclose(out["grad"], cs, rtol=1e-11, atol=1e-13 * np.abs(cs).max())
    # eps(x, y) really is the second output: the loss moves with its bias
    assert abs(cs[-1]) > 1e-6
