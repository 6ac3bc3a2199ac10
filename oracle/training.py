"""Loss, gradients, meta network and optimiser for neural-solver training (oracle; test only).

Algorithm 1 of the paper: weights w = Meta(theta; mu); unroll K iterations of the
Table 1 method from u0; loss L2 of eq. 15; backpropagate. Readings used here:
  * the loss is the mean *log* relative residual (1/B) sum_b ln(||f_b - A_b u_b^K|| / ||f_b||)
    (a monotone transform of eq. 15 per instance; natural log);
  * the meta network is an MLP 2 -> 64 -> 64 -> (m+1) with ReLU, inputs (log10 eps, theta)
    (Sec. 2.4 feeds lg eps); outputs o map to w_i = exp(o_i) / G (G the Gershgorin bound
    of the instance, so the net predicts scale-free log-weights, cf. the log-w
    parametrisation of Sec. 3.2) and a momentum a = sigmoid(o_m) shared by all m steps;
  * the NAG form (at = a), zero initial velocity.
Gradients are taken by PyTorch autograd (FP64, CPU) through a plain forward that
multiplies by the element-assembled sparse matrix; they are pinned by central finite
differences of the same forward (tests).
"""
from __future__ import annotations

import warnings

import numpy as np
import torch

warnings.filterwarnings("ignore", message="Sparse CSR tensor support is in beta state")
warnings.filterwarnings("ignore", message="Sparse invariant checks are implicitly disabled")


def to_torch_sparse(A):
    """scipy CSR -> torch CSR (float64 or complex128), CPU."""
    A = A.tocsr()
    return torch.sparse_csr_tensor(torch.from_numpy(A.indptr.astype(np.int64)),
                                   torch.from_numpy(A.indices.astype(np.int64)),
                                   torch.from_numpy(A.data), size=A.shape)


def unrolled_nag(At, f, u0, w, a, K, Dinv=None, Binv=None, at=None):
    """K inner steps of Table 1's NAGex form in torch; u^{-1} = u0 (zero velocity).

    w, a: tensors of length m (a may be a length-m tensor or a scalar tensor).
    at: the look-ahead momenta (length m), or None for at = a (NAG); zeros give MOM,
    and a = at = 0 Richardson(m).
    Dinv: optional tensor, elementwise B^{-1} = D^{-1} (eq. 17).
    Binv: optional dense tensor, B^{-1} as a matrix (e.g. the SSOR preconditioner).
    """
    m = w.shape[0]
    u = u0
    v = torch.zeros_like(u0)
    for k in range(K):
        i = k % m
        ai = a[i] if a.dim() > 0 else a
        ati = ai if at is None else at[i]
        ut = u + ati * v
        r = f - At @ ut
        if Dinv is not None:
            r = Dinv * r
        if Binv is not None:
            r = Binv @ r
        v = ai * v + w[i] * r
        u = u + v
    return u


def log_rel_residual(At, f, u):
    """ln(||f - A u|| / ||f||)."""
    return torch.log(torch.linalg.vector_norm(f - At @ u) / torch.linalg.vector_norm(f))


def loss_and_grads(As, fs, u0s, ws, alphas, K, Dinvs=None, Binvs=None):
    """Mean log relative residual after K NAG steps and its gradient.

    As: list of scipy matrices; fs, u0s: lists of flat numpy arrays; ws: (B, m);
    alphas: (B, m) per-step momentum or (B,) one momentum per instance.
    Dinvs: optional per-instance diagonals of D^{-1}; Binvs: optional per-instance
    dense B^{-1} matrices (oracle.iterations.ssor_binv_matrix).
    Returns (L, dL/dw (B, m), dL/dalpha (same shape as alphas), [dL/du0_b]).
    Pinned by: central finite differences (tests).
    """
    B = len(As)
    w_t = torch.tensor(np.asarray(ws, dtype=np.float64), requires_grad=True)
    a_t = torch.tensor(np.asarray(alphas, dtype=np.float64), requires_grad=True)
    u0_t = [torch.tensor(np.asarray(u, dtype=np.float64), requires_grad=True) for u in u0s]
    total = 0.0
    for b in range(B):
        At = to_torch_sparse(As[b])
        f = torch.from_numpy(np.asarray(fs[b], dtype=np.float64))
        Dinv = None if Dinvs is None else torch.from_numpy(np.asarray(Dinvs[b]))
        Binv = None if Binvs is None else torch.from_numpy(np.asarray(Binvs[b], dtype=np.float64))
        uK = unrolled_nag(At, f, u0_t[b], w_t[b], a_t[b], K, Dinv, Binv)
        total = total + log_rel_residual(At, f, uK)
    L = total / B
    L.backward()
    return float(L.detach()), w_t.grad.numpy(), a_t.grad.numpy(), [u.grad.numpy() for u in u0_t]


def loss_only(As, fs, u0s, ws, alphas, K, Binvs=None):
    """The same loss without gradients (used for finite differences)."""
    with torch.no_grad():
        tot = 0.0
        for b in range(len(As)):
            At = to_torch_sparse(As[b])
            f = torch.from_numpy(np.asarray(fs[b], dtype=np.float64))
            uK = unrolled_nag(At, f, torch.tensor(np.asarray(u0s[b], dtype=np.float64)),
                              torch.tensor(np.asarray(ws[b], dtype=np.float64)),
                              torch.tensor(np.asarray(alphas[b], dtype=np.float64)), K,
                              Binv=None if Binvs is None else torch.from_numpy(np.asarray(Binvs[b],
                                                                                           dtype=np.float64)))
            tot += float(log_rel_residual(At, f, uK))
    return tot / len(As)


def loss_and_grads_general(As, fs, u0s, ws, alphas, alpha_ts, K):
    """The mean log relative residual after K steps of Table 1's NAGex form (at = None:
    NAG; alphas = None: Richardson(m)) for real or complex states (the Helmholtz
    operators: As complex scipy matrices, fs and u0s complex arrays, real weights), and
    its gradients (dL/dw, dL/dalpha, dL/dalpha_t (B, m) each or None, [dL/du0_b]). For a
    complex u0 the gradient is dL/dRe u0 + i dL/dIm u0, PyTorch's convention for a real
    function of complex leaves. Pinned by: central finite differences of the same
    forward in every weight and in the real and imaginary parts of u0 (tests)."""
    B = len(As)
    w_t = torch.tensor(np.asarray(ws, dtype=np.float64), requires_grad=True)
    a_t = None if alphas is None else torch.tensor(np.asarray(alphas, dtype=np.float64), requires_grad=True)
    at_t = None if alpha_ts is None else torch.tensor(np.asarray(alpha_ts, dtype=np.float64), requires_grad=True)
    u0_t = [torch.tensor(np.asarray(u), requires_grad=True) for u in u0s]
    total = 0.0
    for b in range(B):
        At = to_torch_sparse(As[b])
        f = torch.from_numpy(np.asarray(fs[b]))
        a_b = torch.zeros_like(w_t[b]) if a_t is None else a_t[b]
        uK = unrolled_nag(At, f, u0_t[b], w_t[b], a_b, K, at=None if at_t is None else at_t[b])
        total = total + log_rel_residual(At, f, uK)
    L = total / B
    L.backward()
    return (float(L.detach()), w_t.grad.numpy(), None if a_t is None else a_t.grad.numpy(),
            None if at_t is None else at_t.grad.numpy(), [u.grad.numpy() for u in u0_t])


def loss_general(As, fs, u0s, ws, alphas, alpha_ts, K):
    """The loss of ``loss_and_grads_general`` by the numpy iteration of
    ``oracle.iterations.inner_steps`` (no autograd; for finite differences)."""
    from oracle.iterations import inner_steps
    tot = 0.0
    for b in range(len(As)):
        u, _ = inner_steps(As[b], fs[b], u0s[b], None, ws[b], None if alphas is None else alphas[b],
                           None if alpha_ts is None else alpha_ts[b], K=K)
        tot += np.log(np.linalg.norm(fs[b] - As[b] @ u) / np.linalg.norm(fs[b]))
    return tot / len(As)


# ---------------------------------------------------------------- meta network

def mlp_forward(params, X):
    """o = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X (numpy, FP64).

    params: [(W1, b1), (W2, b2), (W3, b3)], W[out][in]. Pinned by: a hand-evaluated
    2-2-2-1 network (tests).
    """
    h = np.asarray(X, dtype=np.float64)
    for li, (W, b) in enumerate(params):
        h = h @ np.asarray(W).T + np.asarray(b)
        if li < len(params) - 1:
            h = np.maximum(h, 0.0)
    return h


def meta_output_map(o, G, m):
    """w_i = exp(o_i) / G (i < m), a = sigmoid(o_m) (reading; see module docstring)."""
    o = np.asarray(o, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64).reshape(-1, 1)
    w = np.exp(o[:, :m]) / G
    a = 1.0 / (1.0 + np.exp(-o[:, m]))
    return w, a


# Output heads of the meta network: which Table 1 method its outputs parametrise.
HEAD_NAG_SHARED, HEAD_RICHARDSON, HEAD_MOM, HEAD_NAG, HEAD_NAGEX = 0, 1, 2, 3, 4


def head_outputs(head, m):
    """Number of network outputs of a head: m weights, plus one shared momentum (NAG
    with a single a), m per-step momenta (MOM, NAG) or 2m (NAGex: a_i and at_i)."""
    return {HEAD_NAG_SHARED: m + 1, HEAD_RICHARDSON: m, HEAD_MOM: 2 * m, HEAD_NAG: 2 * m, HEAD_NAGEX: 3 * m}[head]


def head_map(o, G, m, head):
    """(w, a, at), each (B, m), from network outputs o (B, head_outputs) in torch:
    w_i = exp(o_i) / G; a_i = sigmoid of the momentum output(s); at per Table 1's row
    (NAG: at = a; MOM: 0; NAGex: its own outputs; Richardson: a = at = 0)."""
    B = o.shape[0]
    w = torch.exp(o[:, :m]) / G.reshape(-1, 1)
    zero = torch.zeros(B, m, dtype=o.dtype)
    if head == HEAD_RICHARDSON:
        return w, zero, zero
    if head == HEAD_NAG_SHARED:
        a = torch.sigmoid(o[:, m]).reshape(-1, 1).expand(B, m)
        return w, a, a
    a = torch.sigmoid(o[:, m:2 * m])
    if head == HEAD_MOM:
        return w, a, zero
    if head == HEAD_NAG:
        return w, a, a
    return w, a, torch.sigmoid(o[:, 2 * m:3 * m])


def mlp_loss_and_grads(params, X, G, m, As, fs, K, head=HEAD_NAG_SHARED, Binvs=None):
    """Training loss of Algorithm 1 (x0 = 0, K steps of the head's Table 1 method,
    optionally with dense B^{-1} matrices) and its gradient wrt the MLP.

    Returns (L, [(dW, db) per layer], w (B, m), a): a is (B,) for the shared-momentum
    head, else the (B, m) momenta. Pinned by: finite differences.
    """
    tp = [(torch.tensor(np.asarray(W, dtype=np.float64), requires_grad=True),
           torch.tensor(np.asarray(b, dtype=np.float64), requires_grad=True)) for W, b in params]
    h = torch.from_numpy(np.asarray(X, dtype=np.float64))
    for li, (W, b) in enumerate(tp):
        h = h @ W.T + b
        if li < len(tp) - 1:
            h = torch.relu(h)
    Gt = torch.from_numpy(np.asarray(G, dtype=np.float64))
    w, a, at = head_map(h, Gt, m, head)
    total = 0.0
    for b in range(len(As)):
        At = to_torch_sparse(As[b])
        f = torch.from_numpy(np.asarray(fs[b], dtype=np.float64))
        Binv = None if Binvs is None else torch.from_numpy(np.asarray(Binvs[b], dtype=np.float64))
        uK = unrolled_nag(At, f, torch.zeros_like(f), w[b], a[b], K, Binv=Binv, at=at[b])
        total = total + log_rel_residual(At, f, uK)
    L = total / len(As)
    L.backward()
    grads = [(W.grad.numpy(), b.grad.numpy()) for W, b in tp]
    a_out = a[:, 0] if head == HEAD_NAG_SHARED else a
    return float(L.detach()), grads, w.detach().numpy(), a_out.detach().numpy()


def adam_step(p, g, m1, m2, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015) on arrays; returns (p, m1, m2). t is 1-based."""
    m1 = b1 * m1 + (1.0 - b1) * g
    m2 = b2 * m2 + (1.0 - b2) * g * g
    mh = m1 / (1.0 - b1 ** t)
    vh = m2 / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
