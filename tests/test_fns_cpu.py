"""Host logic of the Richardson(m)-FNS module (Sec. 3.1)."""
import numpy as np


def test_periodic_inverse_symbol_inverts_the_circulant_stencil():
    # S from paper_2412_08076_gb300.fns against the periodic (circulant) matrix of the
    # oracle's interior Q1 row: P ifft2(S fft2(r)) = r for mean-free r
    from oracle.operators import assemble_q1
    from paper_2412_08076_gb300 import fns
    n = 9
    for eps, th in [(1e-2, 0.7), (1.0, 2.2), (1e-4, 0.1)]:
        A = assemble_q1(n, eps, th).toarray()
        h = n // 2
        row = A[h * n + h].reshape(n, n)
        coef = [row[h, h], row[h, h + 1], row[h + 1, h], row[h + 1, h + 1], row[h + 1, h - 1]]
        S = fns.periodic_inverse_symbol(coef, n, delta=1e-13)
        P = np.zeros((n * n, n * n))
        for a in range(n):
            for b in range(n):
                for di in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        P[a * n + b, ((a + di) % n) * n + (b + dj) % n] += row[h + di, h + dj]
        r = np.random.default_rng(1).standard_normal((n, n))
        r -= r.mean()
        x = np.fft.ifft2(S * np.fft.fft2(r)).real
        np.testing.assert_allclose(P @ x.ravel(), r.ravel(), atol=1e-9)
