"""Pins of the oracle's gradients, meta network, optimiser and Fourier correction."""
import math

import numpy as np

import richm_synth as synth
from oracle.fourier import fourier_correction, fourier_correction_vjp, two_level_cycle
from oracle.iterations import inner_steps, semi_iteration_weights
from oracle.operators import assemble_q1, gershgorin_max
from oracle.training import (adam_step, loss_and_grads, loss_only, meta_output_map,
                             mlp_forward, mlp_loss_and_grads)


def _problem(B=2, n=7, K=12, m=4):
    As, fs, u0s = [], [], []
    for b in range(B):
        A = assemble_q1(n, [1e-2, 0.3, 1.0][b % 3], [0.4, 2.0, 1.1][b % 3])
        As.append(A)
        fs.append(synth.rhs_uniform(21, b, n).ravel())
        u0s.append(0.1 * synth.rhs_uniform(22, b, n).ravel())
    w = np.stack([semi_iteration_weights(gershgorin_max(A), m) * 0.5 for A in As])
    a = np.full((B, m), 0.3) + 0.05 * np.arange(m)
    return As, fs, u0s, w, a, K


def test_loss_gradient_matches_central_differences():
    As, fs, u0s, w, a, K = _problem()
    L, gw, ga, gu = loss_and_grads(As, fs, u0s, w, a, K)
    h = 1e-4
    for b in range(2):
        for i in range(w.shape[1]):
            wp, wm = w.copy(), w.copy()
            wp[b, i] += h
            wm[b, i] -= h
            fd = (loss_only(As, fs, u0s, wp, a, K) - loss_only(As, fs, u0s, wm, a, K)) / (2 * h)
            assert abs(fd - gw[b, i]) <= 1e-6 * max(1.0, abs(fd)), (b, i, fd, gw[b, i])
            ap, am = a.copy(), a.copy()
            ap[b, i] += h
            am[b, i] -= h
            fd = (loss_only(As, fs, u0s, w, ap, K) - loss_only(As, fs, u0s, w, am, K)) / (2 * h)
            assert abs(fd - ga[b, i]) <= 1e-6 * max(1.0, abs(fd))
        for idx in [0, 11, 24, 48]:
            up = [u.copy() for u in u0s]
            um = [u.copy() for u in u0s]
            up[b][idx] += h
            um[b][idx] -= h
            fd = (loss_only(As, fs, up, w, a, K) - loss_only(As, fs, um, w, a, K)) / (2 * h)
            assert abs(fd - gu[b][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_loss_value_is_mean_log_relative_residual():
    As, fs, u0s, w, a, K = _problem()
    L = loss_only(As, fs, u0s, w, a, K)
    ref = 0.0
    for b in range(2):
        u, _ = inner_steps(As[b], fs[b], u0s[b], None, w[b], a[b], K=K)
        ref += math.log(np.linalg.norm(fs[b] - As[b] @ u) / np.linalg.norm(fs[b]))
    assert abs(L - ref / 2) < 1e-12


def test_mlp_forward_hand_evaluated():
    # 2-2-2-1 network evaluated by hand
    params = [(np.array([[1.0, -1.0], [0.5, 2.0]]), np.array([0.0, -1.0])),
              (np.array([[1.0, 1.0], [-1.0, 3.0]]), np.array([0.5, 0.0])),
              (np.array([[2.0, -1.0]]), np.array([0.25]))]
    X = np.array([[1.0, 2.0], [3.0, -1.0]])
    # x=(1,2): h1=relu(-1, 3.5)=(0,3.5); h2=relu(4, 10.5)=(4,10.5); o=8-10.5+0.25=-2.25
    # x=(3,-1): h1=relu(4,-1.5)=(4,0); h2=relu(4.5,-4)=(4.5,0); o=9+0.25=9.25
    np.testing.assert_allclose(mlp_forward(params, X), [[-2.25], [9.25]])
    w, a = meta_output_map(np.array([[0.0, math.log(2.0), 0.0]]), [4.0], 2)
    np.testing.assert_allclose(w, [[0.25, 0.5]])
    np.testing.assert_allclose(a, [0.5])


def test_mlp_training_gradient_matches_central_differences():
    m, K, n = 4, 10, 6
    params = synth.mlp_init((2, 8, 8, m + 1), seed=3)
    params = [(W * 0.3, b * 0.3) for W, b in params]
    insts = [synth.AnisoInstance(1e-2, 0.5, n), synth.AnisoInstance(0.5, 2.0, n)]
    As = [assemble_q1(n, t.eps, t.theta) for t in insts]
    G = np.array([gershgorin_max(A) for A in As])
    fs = [synth.rhs_uniform(5, b, n).ravel() for b in range(2)]
    X = synth.meta_inputs(insts)
    L, grads, _, _ = mlp_loss_and_grads(params, X, G, m, As, fs, K)
    h = 1e-5
    rng = np.random.default_rng(0)
    for li in range(3):
        W, b = params[li]
        for _ in range(3):
            r, c = rng.integers(0, W.shape[0]), rng.integers(0, W.shape[1])
            vals = []
            for sgn in (1, -1):
                P = [(Wk.copy(), bk.copy()) for Wk, bk in params]
                P[li][0][r, c] += sgn * h
                vals.append(mlp_loss_and_grads(P, X, G, m, As, fs, K)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grads[li][0][r, c]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m1, m2 = adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=1e-14)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(m2, 0.001 * g * g)


def test_fft_matches_explicit_dft_and_zero_symbol():
    for n in [5, 12, 33]:
        A = assemble_q1(n, 1e-2, 1.0)
        f = synth.rhs_uniform(9, n, n).ravel()
        u = 0.3 * synth.rhs_uniform(8, n, n).ravel()
        S = synth.fourier_symbol(n, seed=3)
        jj = np.arange(n)
        F = np.exp(-2j * math.pi * np.outer(jj, jj) / n)
        r = (f - A @ u).reshape(n, n)
        c = (F.conj() @ (S * (F @ r @ F.T)) @ F.conj().T) / (n * n)
        np.testing.assert_allclose(fourier_correction(A, f, u, S), u + c.real.ravel(), atol=1e-12)
        np.testing.assert_array_equal(fourier_correction(A, f, u, np.zeros((n, n))), u)


def _vjp_case(n, seed):
    A = assemble_q1(n, [1e-2, 1e-4][n % 2], 0.7 + 0.2 * n)
    f = synth.rhs_uniform(9, seed, n).ravel()
    u = 0.3 * synth.rhs_uniform(8, seed, n).ravel()
    S = synth.fourier_symbol(n, seed=seed)
    g = synth.rhs_uniform(7, seed, n).ravel()
    return A, f, u, S, g


def test_fourier_vjp_matches_central_differences():
    # <g, u'> is linear in S and affine in u, so central differences are exact up to
    # rounding: a dropped conjugate, a transposed spectrum or a lost 1/n^2 fails here
    for n in (5, 6):
        A, f, u, S, g = _vjp_case(n, 11 + n)
        dS, du = fourier_correction_vjp(A, f, u, S, g)
        L = lambda uu, SS: g @ fourier_correction(A, f, uu, SS)
        h = 1e-6
        for k1 in range(n):
            for k2 in range(n):
                E = np.zeros((n, n))
                E[k1, k2] = 1.0
                re = (L(u, S + h * E) - L(u, S - h * E)) / (2 * h)
                im = (L(u, S + 1j * h * E) - L(u, S - 1j * h * E)) / (2 * h)
                assert abs(re + 1j * im - dS[k1, k2]) < 1e-8
        fdu = np.array([(L(u + h * e, S) - L(u - h * e, S)) / (2 * h) for e in np.eye(n * n)])
        np.testing.assert_allclose(du, fdu, atol=1e-8)


def test_fourier_vjp_matches_autograd_and_is_hermitian():
    import torch
    n = 8
    A, f, u, S, g = _vjp_case(n, 4)
    dS, du = fourier_correction_vjp(A, f, u, S, g)
    At = torch.tensor(A.toarray())
    St = torch.tensor(S, requires_grad=True)
    ut = torch.tensor(u, requires_grad=True)
    r = (torch.tensor(f) - At @ ut).reshape(n, n)
    up = ut + torch.fft.ifft2(St * torch.fft.fft2(r)).real.reshape(-1)
    (torch.tensor(g) * up).sum().backward()
    np.testing.assert_allclose(dS, St.grad.numpy(), atol=1e-13)
    np.testing.assert_allclose(du, ut.grad.numpy(), atol=1e-13)
    # real r and g: dS(-k) = conj(dS(k))
    idx = (-np.arange(n)) % n
    np.testing.assert_allclose(dS[np.ix_(idx, idx)], np.conj(dS), atol=1e-13)


def test_two_level_exact_inverse_symbol_on_periodic_free_case():
    # With S = 0 a cycle is plain Richardson(m).
    n = 9
    A = assemble_q1(n, 1e-2, 0.3)
    f = synth.rhs_uniform(1, 0, n).ravel()
    w = semi_iteration_weights(gershgorin_max(A), 8)
    u1 = two_level_cycle(A, f, np.zeros(n * n), w, np.zeros((n, n)))
    u2, _ = inner_steps(A, f, np.zeros(n * n), None, w, K=8)
    np.testing.assert_array_equal(u1, u2)


def test_ssor_preconditioned_loss_and_gradient():
    # forward: the dense-B^{-1} unroll equals the Table 1 steps with the SSOR solves as
    # triangular-solve callables; gradient: central differences of that forward
    from oracle.iterations import ssor_binv, ssor_binv_matrix
    As, fs, u0s, w, a, K = _problem(n=6, K=8)
    relax = 1.4
    Bm = [ssor_binv_matrix(A, relax) for A in As]
    w = w * 2.0  # B^{-1} A has its spectrum in (0, 1]: weights of order 1
    L, gw, ga, gu = loss_and_grads(As, fs, u0s, w, a, K, Binvs=Bm)
    ref = 0.0
    for b in range(2):
        u, _ = inner_steps(As[b], fs[b], u0s[b], None, w[b], a[b], K=K, Binv=ssor_binv(As[b], relax))
        ref += math.log(np.linalg.norm(fs[b] - As[b] @ u) / np.linalg.norm(fs[b]))
    assert abs(L - ref / 2) < 1e-12
    h = 1e-5
    for b in range(2):
        for i in range(w.shape[1]):
            for arr, g in ((w, gw), (a, ga)):
                p, q = arr.copy(), arr.copy()
                p[b, i] += h
                q[b, i] -= h
                args_p = (p, a) if arr is w else (w, p)
                args_q = (q, a) if arr is w else (w, q)
                fd = (loss_only(As, fs, u0s, *args_p, K, Binvs=Bm) - loss_only(As, fs, u0s, *args_q, K, Binvs=Bm)) / (2 * h)
                assert abs(fd - g[b, i]) <= 1e-6 * max(1.0, abs(fd)), (b, i, fd, g[b, i])
        for idx in [0, 7, 20, 35]:
            up = [u.copy() for u in u0s]
            um = [u.copy() for u in u0s]
            up[b][idx] += h
            um[b][idx] -= h
            fd = (loss_only(As, fs, up, w, a, K, Binvs=Bm) - loss_only(As, fs, um, w, a, K, Binvs=Bm)) / (2 * h)
            assert abs(fd - gu[b][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_ssor_binv_matrix_is_the_operator():
    from oracle.iterations import ssor_binv, ssor_binv_matrix
    A = assemble_q1(5, 0.05, 0.7)
    M = ssor_binv_matrix(A, 1.2)
    r = synth.rhs_uniform(5, 0, 5).ravel()
    np.testing.assert_allclose(M @ r, ssor_binv(A, 1.2)(r), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(M, M.T, atol=1e-14 * np.abs(M).max())


def test_head_map_hand_evaluated():
    import torch
    from oracle.training import (HEAD_MOM, HEAD_NAG, HEAD_NAG_SHARED, HEAD_NAGEX, HEAD_RICHARDSON, head_map,
                                 head_outputs)
    m = 2
    assert [head_outputs(h, m) for h in range(5)] == [3, 2, 4, 4, 6]
    L2, L3 = math.log(2.0), math.log(3.0)  # sigmoid(ln 3) = 3/4, sigmoid(-ln 3) = 1/4
    o = torch.tensor([[0.0, L2, L3, -L3, 0.0, L3]], dtype=torch.float64)
    G = torch.tensor([4.0], dtype=torch.float64)
    expect = {
        HEAD_RICHARDSON: ([0.25, 0.5], [0, 0], [0, 0]),
        HEAD_NAG_SHARED: ([0.25, 0.5], [0.75, 0.75], [0.75, 0.75]),
        HEAD_MOM: ([0.25, 0.5], [0.75, 0.25], [0, 0]),
        HEAD_NAG: ([0.25, 0.5], [0.75, 0.25], [0.75, 0.25]),
        HEAD_NAGEX: ([0.25, 0.5], [0.75, 0.25], [0.5, 0.75]),
    }
    for head, (we, ae, ate) in expect.items():
        w, a, at = head_map(o[:, :head_outputs(head, m)], G, m, head)
        np.testing.assert_allclose(w.numpy(), [we], rtol=1e-15)
        np.testing.assert_allclose(a.numpy(), [ae], rtol=1e-15)
        np.testing.assert_allclose(at.numpy(), [ate], rtol=1e-15)


def test_unrolled_with_lookahead_momenta_matches_inner_steps():
    # the torch unroll with separate at equals the Table 1 steps of the numpy oracle
    import torch
    from oracle.training import to_torch_sparse, unrolled_nag
    As, fs, u0s, w, a, K = _problem(B=1, n=6, K=11, m=3)
    at = np.array([0.1, 0.6, 0.35])
    for at_ in (at, np.zeros(3)):
        u = unrolled_nag(to_torch_sparse(As[0]), torch.from_numpy(fs[0]), torch.from_numpy(u0s[0]),
                         torch.from_numpy(w[0]), torch.from_numpy(a[0]), K, at=torch.from_numpy(at_))
        ref, _ = inner_steps(As[0], fs[0], u0s[0], None, w[0], a[0], at_, K=K)
        np.testing.assert_allclose(u.numpy(), ref, rtol=1e-13, atol=1e-15)


def test_head_training_gradients_match_central_differences():
    # every head, and the NAGex head through a dense SSOR B^{-1}
    from oracle.iterations import ssor_binv_matrix
    from oracle.training import HEAD_MOM, HEAD_NAGEX, HEAD_RICHARDSON, head_outputs
    m, K, n = 3, 9, 5
    insts = [synth.AnisoInstance(1e-2, 0.5, n), synth.AnisoInstance(0.5, 2.0, n)]
    As = [assemble_q1(n, t.eps, t.theta) for t in insts]
    fs = [synth.rhs_uniform(5, b, n).ravel() for b in range(2)]
    X = synth.meta_inputs(insts)
    rng = np.random.default_rng(1)
    for head, ssor in ((HEAD_RICHARDSON, False), (HEAD_MOM, False), (HEAD_NAGEX, False), (HEAD_NAGEX, True)):
        params = synth.mlp_init((2, 6, 6, head_outputs(head, m)), seed=4)
        params = [(W * 0.3, b * 0.3) for W, b in params]
        Bm = [ssor_binv_matrix(A, 1.2) for A in As] if ssor else None
        G = np.ones(2) if ssor else np.array([gershgorin_max(A) for A in As])
        L, grads, _, _ = mlp_loss_and_grads(params, X, G, m, As, fs, K, head=head, Binvs=Bm)
        h = 1e-5
        for li in range(3):
            W, b = params[li]
            r, c = rng.integers(0, W.shape[0]), rng.integers(0, W.shape[1])
            vals = []
            for sgn in (1, -1):
                P = [(Wk.copy(), bk.copy()) for Wk, bk in params]
                P[li][0][r, c] += sgn * h
                vals.append(mlp_loss_and_grads(P, X, G, m, As, fs, K, head=head, Binvs=Bm)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grads[li][0][r, c]) <= 1e-6 * max(1.0, abs(fd)), (head, ssor, li, fd)


def _band_kernel(w, seed):
    """A Hermitian-symmetric (2w+1)^2 band kernel: tau[-d] = conj(tau[d])."""
    rng = np.random.default_rng(seed)
    k = 2 * w + 1
    tau = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    tau = 0.5 * (tau + np.conj(tau[::-1, ::-1]))
    tau[w, w] = 1.0 + 0.0j
    return 0.3 * tau


def test_transition_correction_equals_the_matrix_product():
    # H = F T S T^H F^{-1} written out: DFT matrices for the transforms, T the banded
    # matrix T[k, k'] = tau[k - k'] (indices mod n) acting on the spectrum, S diagonal
    from oracle.fourier import fourier_correction, fourier_correction_t, transition_field
    from oracle.operators import assemble_q1
    for n, w in [(6, 1), (7, 2), (5, 1)]:
        A = assemble_q1(n, 0.1, 0.6)
        rng = np.random.default_rng(n)
        f, u = rng.standard_normal(n * n), rng.standard_normal(n * n)
        S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        tau = _band_kernel(w, n)
        j = np.arange(n)
        D1 = np.exp(-2j * np.pi * np.outer(j, j) / n)
        Fwd = np.kron(D1, D1)                    # fft2 on row-major flattening
        Inv = np.conj(Fwd) / (n * n)             # ifft2
        T = np.zeros((n * n, n * n), complex)
        for k1 in range(n):
            for k2 in range(n):
                for a in range(-w, w + 1):
                    for c in range(-w, w + 1):
                        T[k1 * n + k2, ((k1 - a) % n) * n + (k2 - c) % n] += tau[a + w, c + w]
        H = Inv @ T @ np.diag(S.ravel()) @ T.conj().T @ Fwd
        ref = u + (H @ (f - A @ u)).real
        got = fourier_correction_t(A, f, u, S, transition_field(tau, n))
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)
        # the identity transition is the plain correction
        np.testing.assert_allclose(fourier_correction_t(A, f, u, S, np.ones((n, n))),
                                   fourier_correction(A, f, u, S), rtol=1e-13, atol=1e-13)


def test_transition_vjp_matches_central_differences():
    from oracle.fourier import fourier_correction_t, fourier_correction_t_vjp, transition_field
    from oracle.operators import assemble_q1
    n = 6
    A = assemble_q1(n, 0.05, 1.1)
    rng = np.random.default_rng(9)
    f, u, g = rng.standard_normal(n * n), rng.standard_normal(n * n), rng.standard_normal(n * n)
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    t = transition_field(_band_kernel(1, 3), n)
    dS, dt, du = fourier_correction_t_vjp(A, f, u, S, t, g)

    def L(S_, t_, u_):
        return float(np.dot(g, fourier_correction_t(A, f, u_, S_, t_)))
    h = 1e-6
    for (a, c) in [(0, 0), (2, 5), (4, 1)]:
        E = np.zeros((n, n))
        E[a, c] = h
        assert abs((L(S + E, t, u) - L(S - E, t, u)) / (2 * h) - dS[a, c].real) < 1e-7
        assert abs((L(S + 1j * E, t, u) - L(S - 1j * E, t, u)) / (2 * h) - dS[a, c].imag) < 1e-7
        assert abs((L(S, t + E, u) - L(S, t - E, u)) / (2 * h) - dt[a, c]) < 1e-7
        e = E.ravel()
        assert abs((L(S, t, u + e) - L(S, t, u - e)) / (2 * h) - du[a * n + c]) < 1e-7


def test_symbol_map_is_the_periodic_spectrum_and_has_its_gradient():
    # o = 0 and no regularisation: 1/S is the spectrum of the periodic extension of the Q1
    # operator (a block-circulant matrix built from the stencil), in DFT order
    from oracle.fourier import symbol_from_stencil
    import math
    n = 6
    eps, th = 0.1, 0.7
    c, s = math.cos(th), math.sin(th)
    c11, c22, c12 = c * c + eps * s * s, s * s + eps * c * c, (1 - eps) * s * c
    q = [4 * (c11 + c22) / 3, (c22 - 2 * c11) / 3, (c11 - 2 * c22) / 3,
         -(c11 + c22) / 6 - c12 / 2, -(c11 + c22) / 6 + c12 / 2, 1e-9]
    P = np.zeros((n * n, n * n))
    for i in range(n):
        for j in range(n):
            for (di, dj, v) in [(0, 0, q[0]), (0, -1, q[1]), (0, 1, q[1]), (-1, 0, q[2]), (1, 0, q[2]),
                                (1, 1, q[3]), (-1, -1, q[3]), (-1, 1, q[4]), (1, -1, q[4])]:
                P[i * n + j, ((i + di) % n) * n + (j + dj) % n] += v
    S = symbol_from_stencil(q, np.zeros(6), n)
    # every DFT mode is an eigenvector of the circulant operator with eigenvalue sigma(k),
    # and S = 1/sigma there (the k = 0 mode: sigma = 0, S bounded by 1/(2 delta))
    for k1 in range(n):
        for k2 in range(n):
            v = np.exp(2j * np.pi * (k1 * np.arange(n)[:, None] + k2 * np.arange(n)[None, :]) / n).ravel()
            Pv = P @ v
            if k1 == 0 and k2 == 0:
                assert np.abs(Pv).max() < 1e-12 and abs(S[0, 0]) <= 0.5 / 1e-9  # at most 1/(2 delta)
            else:
                np.testing.assert_allclose(Pv, v / S[k1, k2].real, rtol=1e-9, atol=1e-12)
    # the reverse mode: dL/do for L = Re sum conj(G) S, against central differences
    from oracle.fourier import symbol_from_stencil as sym
    rng = np.random.default_rng(1)
    G = rng.standard_normal((n, n))
    o = 0.1 * rng.standard_normal(6)
    q2 = list(q[:5]) + [0.2]
    h = 1e-6
    for m in range(6):
        e = np.zeros(6)
        e[m] = h
        fd = (np.sum(G * sym(q2, o + e, n).real) - np.sum(G * sym(q2, o - e, n).real)) / (2 * h)
        t = 2.0 * np.pi * np.arange(n) / n
        t1, t2 = np.meshgrid(t, t, indexing="ij")
        p = np.array(q2[:5]) * np.exp(o[:5])
        d = q2[5] * np.exp(o[5])
        basis = [np.ones_like(t1), 2 * np.cos(t2), 2 * np.cos(t1), 2 * np.cos(t1 + t2), 2 * np.cos(t1 - t2)]
        sig = sum(pm * bm for pm, bm in zip(p, basis))
        den = sig ** 2 + d ** 2
        if m < 5:
            an = np.sum(G * (d * d - sig ** 2) / den ** 2 * basis[m] * p[m])
        else:
            an = np.sum(G * (-2 * sig * d) / den ** 2 * d)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_transition_band_parametrisation():
    from oracle.fourier import transition_band, transition_field
    n = 7
    tau9 = np.array([1.0, 0.1, -0.2, 0.05, 0.3, -0.15, 0.02, 0.07, -0.01])
    t = transition_band(tau9, n)
    # written out term by term
    i, j = np.arange(n)[:, None], np.arange(n)[None, :]
    ref = tau9[0] + 0 * i * j
    for q, (a, c) in enumerate([(0, 1), (1, 0), (1, 1), (1, -1)]):
        ang = 2 * np.pi * (a * i + c * j) / n
        ref = ref + 2 * (tau9[1 + 2 * q] * np.cos(ang) - tau9[2 + 2 * q] * np.sin(ang))
    np.testing.assert_allclose(t, ref, atol=1e-12)
    assert np.isrealobj(t)


def _helmholtz_problem(B=2, n=7, K=10, m=4):
    from oracle.operators import assemble_helmholtz, assemble_helmholtz_sponge, helmholtz_wavenumber
    As, fs, u0s = [], [], []
    for b in range(B):
        if b % 2 == 0:
            A = assemble_helmholtz_sponge(n, 2 * math.pi * 1.5)
        else:
            A = assemble_helmholtz(n, helmholtz_wavenumber(n, 6.0), absorbing=True)
        As.append(A.tocsr())
        fs.append(synth.rhs_uniform(31, b, n).ravel() + 1j * synth.rhs_uniform(32, b, n).ravel())
        u0s.append(0.1 * (synth.rhs_uniform(33, b, n).ravel() - 0.5j * synth.rhs_uniform(34, b, n).ravel()))
    G = np.array([abs(A).sum(axis=1).max() for A in As])
    rng = np.random.default_rng(3)
    w = rng.uniform(0.3, 1.2, (B, m)) / G[:, None]
    a = rng.uniform(0.1, 0.4, (B, m))
    at = rng.uniform(0.0, 0.5, (B, m))
    return As, fs, u0s, w, a, at, K


def test_complex_lookahead_gradient_matches_central_differences():
    # complex states (Helmholtz with a sponge layer and with an absorbing boundary),
    # real weights, distinct a and at: every weight and the real and imaginary parts of
    # x0 against central differences of the numpy iteration
    from oracle.training import loss_and_grads_general, loss_general
    As, fs, u0s, w, a, at, K = _helmholtz_problem()
    L, gw, ga, gat, gu = loss_and_grads_general(As, fs, u0s, w, a, at, K)
    assert abs(L - loss_general(As, fs, u0s, w, a, at, K)) < 1e-12
    h = 1e-6
    for name, arr, g in (("w", w, gw), ("a", a, ga), ("at", at, gat)):
        for b in range(2):
            for i in range(w.shape[1]):
                hp = h * max(1.0, abs(arr[b, i]))
                P, M = arr.copy(), arr.copy()
                P[b, i] += hp
                M[b, i] -= hp
                args_p = {"w": (P, a, at), "a": (w, P, at), "at": (w, a, P)}[name]
                args_m = {"w": (M, a, at), "a": (w, M, at), "at": (w, a, M)}[name]
                fd = (loss_general(As, fs, u0s, *args_p, K) - loss_general(As, fs, u0s, *args_m, K)) / (2 * hp)
                scale = max(abs(fd), 1e-3 * np.abs(g).max())
                assert abs(fd - g[b, i]) <= 1e-5 * scale, (name, b, i, fd, g[b, i])
    for b in range(2):
        for idx in (0, 10, 24, 48):
            for unit in (1.0, 1j):
                up = [u.copy() for u in u0s]
                um = [u.copy() for u in u0s]
                up[b][idx] += h * unit
                um[b][idx] -= h * unit
                fd = (loss_general(As, fs, up, w, a, at, K) - loss_general(As, fs, um, w, a, at, K)) / (2 * h)
                comp = gu[b][idx].real if unit == 1.0 else gu[b][idx].imag
                assert abs(fd - comp) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gu[b]).max()), (b, idx, unit, fd, comp)


def test_general_loss_reduces_to_the_real_nag_and_richardson_forms():
    from oracle.training import loss_and_grads_general
    As, fs, u0s, w, a, K = _problem()
    L, gw, ga, gu = loss_and_grads(As, fs, u0s, w, a, K)
    L2, gw2, ga2, gat2, gu2 = loss_and_grads_general(As, fs, u0s, w, a, None, K)
    assert gat2 is None and abs(L - L2) < 1e-13
    np.testing.assert_allclose(gw2, gw, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(ga2, ga, rtol=1e-11, atol=1e-13)
    # Richardson(m): alphas None equals zero momentum
    L3, gw3, ga3, _, _ = loss_and_grads_general(As, fs, u0s, w, None, None, K)
    L4, gw4, _, _ = loss_and_grads(As, fs, u0s, w, np.zeros_like(a), K)
    assert ga3 is None and abs(L3 - L4) < 1e-13
    np.testing.assert_allclose(gw3, gw4, rtol=1e-11, atol=1e-13)
