"""Learned coarse basis (oracle, FP64): input map, labels, loss, a plain
perceptron with its backward pass, and the Rayleigh-Ritz selection that turns
predicted face-flux profiles into coarse basis functions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The method builds its coarse space from one local spectral problem per coarse
face E_i (Section 4.2, eqs. spectral_1 / spectral_eqn) posed on the snapshot
space of eq. snapshot_eqn.  The snapshot v_l^i has normal component delta_l on
the fine faces e_l of E_i, so a coefficient vector over the snapshots is the
normal-velocity profile of the function on those b fine faces: the "flux
profile".  The learned variant predicts, from log kappa on omega_i, k
profiles whose span should contain the eigenfunctions the spectral problem
selects; the profiles are extended to omega_i by the same local solves that
define the snapshots (linearity: one solve per profile), and the spectral
problem is then solved on their span only (Rayleigh-Ritz), keeping the Ritz
values below the tolerance as the spectral selection does.  Where none is
below the tolerance the face falls back to its exact spectral problem.

Readings (the paper has no learned part; these fix the interface):
  * input: log10(kappa) / 3 on omega_i plus a one-cell halo (cells outside
    the domain take the nearest cell's value), in a canonical orientation:
    rows run along E_i, columns across it, K^1 first.  A horizontal coarse
    edge is transposed onto the vertical layout; the flux profile keeps its
    coordinates under the transposition (pinned: the spectral problem of the
    transposed field on the transposed face is the same).
  * coordinates: predictions and labels are "whitened profiles"
    y_l = a_l^{1/2} g_l, g the flux profile and a_l = kappa_e^{-1} the
    diagonal of the a-form on fine face l.  In y the spectral problem is the
    symmetric eigenproblem of D_a^{-1/2} s D_a^{-1/2} (mu = 1/lambda), so a
    subspace at angle theta from its top eigenvectors gives Ritz values within
    O(theta^2); in plain flux coordinates the weights a_l span the contrast
    (1e-6 .. 1e2) and a small Euclidean error on a high-a face ruins the
    Rayleigh quotient.  a is known from kappa, so g = a^{-1/2} y at inference.
  * label: an orthonormal basis (Euclidean, y coordinates) of the span of the
    k eigenfunctions with the smallest eigenvalues (all b when b < k,
    zero-padded).  The span of the lowest modes varies smoothly with kappa,
    unlike the tolerance-selected subset, and it contains every selected
    function when nsel <= k; the tolerance acts at inference, on the Ritz
    values.
  * loss: ||G G^T - Q Q^T||_F^2 per face (G: b x k predicted profiles as
    columns, Q: label), averaged over the batch.  It depends on G only through
    G G^T, so it is invariant under G -> G R for orthogonal R (signs, order,
    rotations of the basis), and it equals the squared Frobenius distance of
    the two orthogonal projectors when G has orthonormal columns.
  * network: x -> relu(W1 x + b1) -> relu(W2 . + b2) -> W3 . + b3, output
    entry j*b + l = profile j at fine face l.
  * selection: directions of span(G) with G^T G eigenvalue above 1/4 (the
    target eigenvalues are 1 and 0), orthonormalised; Ritz pairs of
    a c = lambda s c on that span; keep lambda < tol (at least one); fall
    back to the exact problem when the smallest Ritz value is >= tol, when
    no direction is kept, or when the kept functions carry no net flux
    through E_i (mean profile ~ 0: no unit-flux function can be formed).
"""

import numpy as np
import scipy.linalg as sla

from .coarse import face_blocks, fine_faces_on, jacobi_eigh


# ----------------------------------------------------------------- input map
def input_shape(b):
    """(rows, columns) of the canonical face patch: b + 2 along E_i, 2b + 2 across."""
    return b + 2, 2 * b + 2


def face_input(kappa, g, face):
    """log10(kappa)/3 on omega_i and its one-cell halo, canonical orientation,
    flattened row-major (rows along E_i, columns across it)."""
    kind, I, J = face
    b, n = g.b, g.n
    kap = np.asarray(kappa, float).reshape(n, n)
    R, C = input_shape(b)
    along = np.clip(np.arange(R) - 1 + (J * b if kind == 0 else I * b), 0, n - 1)
    across = np.clip(np.arange(C) - 1 + ((I - 1) * b if kind == 0 else (J - 1) * b), 0, n - 1)
    out = np.empty((R, C))
    for r in range(R):
        for c in range(C):
            cell_val = kap[along[r], across[c]] if kind == 0 else kap[across[c], along[r]]
            out[r, c] = np.log10(cell_val) / 3.0
    return out.ravel()


def face_label(cset, a, k):
    """Orthonormal basis (b x k, zero-padded, y coordinates) of the span of
    the first min(columns, k) coefficient vectors (columns of cset, by
    ascending eigenvalue); a: the a-form diagonal of the face."""
    b, m = cset.shape
    m = min(m, k)
    Q = np.zeros((b, k))
    if m:
        q, _ = np.linalg.qr(np.sqrt(np.asarray(a))[:, None] * cset[:, :m])
        Q[:, :m] = q
    return Q


# ----------------------------------------------------------------- BF16
def bf16(x):
    """Round to the nearest bfloat16 (ties to even), through float32 first as
    a float32 accumulator rounded to bfloat16 would be."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


# ----------------------------------------------------------------- network
def param_layout(b, k, hidden):
    """Names, shapes and offsets of the flat FP32 parameter vector."""
    R, C = input_shape(b)
    din, dout = R * C, k * b
    shapes = [("W1", (hidden, din)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
              ("W3", (dout, hidden)), ("b3", (dout,))]
    out, off = [], 0
    for name, shp in shapes:
        size = int(np.prod(shp))
        out.append((name, shp, off, size))
        off += size
    return out, off


def unpack(flat, b, k, hidden):
    layout, total = param_layout(b, k, hidden)
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == total
    return {name: flat[off:off + size].reshape(shp) for name, shp, off, size in layout}


def pack(p, b, k, hidden):
    layout, total = param_layout(b, k, hidden)
    out = np.zeros(total)
    for name, shp, off, size in layout:
        out[off:off + size] = np.asarray(p[name]).ravel()
    return out


def forward(p, X, emulate_bf16=False):
    """Network output Y (batch x k b) and the values the backward pass needs.
    emulate_bf16 rounds the weights and the hidden activations to bfloat16 at
    the points where the GPU kernels store them in bfloat16."""
    r = bf16 if emulate_bf16 else (lambda v: v)
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    X = np.asarray(X, float)
    H1 = r(np.maximum(X @ W1.T + p["b1"], 0.0))
    H2 = r(np.maximum(H1 @ W2.T + p["b2"], 0.0))
    Y = H2 @ W3.T + p["b3"]
    return Y, (X, H1, H2, W1, W2, W3)


def subspace_loss(Y, Q, b, k):
    """Mean over the batch of ||G G^T - Q Q^T||_F^2 and its gradient dL/dY.
    Y: batch x (k b) with entry j*b + l = G[l, j]; Q: batch x k x b (label
    vectors as rows)."""
    B = Y.shape[0]
    G = Y.reshape(B, k, b).transpose(0, 2, 1)          # B x b x k
    Qc = np.asarray(Q, float).reshape(B, k, b).transpose(0, 2, 1)
    E = G @ G.transpose(0, 2, 1) - Qc @ Qc.transpose(0, 2, 1)
    loss = np.sum(E * E) / B
    dG = (4.0 / B) * (E @ G)                           # d/dG ||G G^T - P||^2 = 4 (G G^T - P) G
    return loss, dG.transpose(0, 2, 1).reshape(B, k * b)


def backward(cache, dY, emulate_bf16=False):
    """Gradients of every parameter given dL/dY (chain rule through the three
    affine maps and the two ReLUs; the ReLU derivative is taken as 1 where the
    stored activation is positive)."""
    r = bf16 if emulate_bf16 else (lambda v: v)
    X, H1, H2, W1, W2, W3 = cache
    dY = r(dY)
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dH2 = r((dY @ W3) * (H2 > 0))
    g["W2"], g["b2"] = dH2.T @ H1, dH2.sum(0)
    dH1 = r((dH2 @ W2) * (H1 > 0))
    g["W1"], g["b1"] = dH1.T @ X, dH1.sum(0)
    return g


def loss_and_grad(flat, X, Q, b, k, hidden, emulate_bf16=False):
    p = unpack(flat, b, k, hidden)
    Y, cache = forward(p, X, emulate_bf16)
    loss, dY = subspace_loss(Y, Q, b, k)
    return loss, pack(backward(cache, dY, emulate_bf16), b, k, hidden)


def adam_step(flat, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), step number t >= 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return flat - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ----------------------------------------------------------------- selection
def ritz_select(G, a, s, tol, thr=0.25):
    """Rayleigh-Ritz form of eq. spectral_eqn on the span of the predicted
    whitened profiles G (b x k, y coordinates).  a: the diagonal of the a-form
    in snapshot coordinates; s: the s-form (b x b).  Returns (Ritz values
    ascending, selected coefficient vectors b x m in snapshot coordinates,
    fallback flag)."""
    w, V = jacobi_eigh(G.T @ G)
    keep = w > thr
    if not keep.any():
        return np.array([]), None, True
    Uy = G @ (V[:, keep] / np.sqrt(w[keep]))          # orthonormal columns (y)
    U = Uy / np.sqrt(np.asarray(a))[:, None]          # flux profiles g = a^{-1/2} y
    ak = U.T @ (np.asarray(a)[:, None] * U)
    sk = U.T @ s @ U
    L = np.linalg.cholesky(0.5 * (ak + ak.T))
    T = sla.solve_triangular(L, sla.solve_triangular(L, sk, lower=True).T, lower=True).T
    mu, Y = jacobi_eigh(0.5 * (T + T.T))
    lam = 1.0 / mu[::-1]
    Y = Y[:, ::-1]
    nsel = max(1, int(np.sum(lam < tol)))
    c = sla.solve_triangular(L.T, Y[:, :nsel], lower=False)
    cset = U @ c
    if lam[0] >= tol:
        return lam, cset, True
    # the kept functions must carry net flux through E_i (the coarse space
    # needs one unit-flux function per face); otherwise fall back
    t = cset.mean(axis=0)
    return lam, cset, bool(np.linalg.norm(t) <= 1e-6 * np.abs(cset).max())


def exact_profiles(g, kappa, tol, k, cap=None):
    """Inputs and labels of every coarse face of one field, from the exact
    spectral problems: (X faces x din, Q faces x k x b, nsel, lam)."""
    from .coarse import BlockSolvers, coarse_faces, snapshots, spectral_problem, solve_spectral
    from .fine import assemble
    kap = np.asarray(kappa, float).reshape(g.n, g.n)
    A, B = assemble(g, kap)
    blocks = BlockSolvers(g, A, B)
    kinv = 1.0 / kap
    X, Q, nsel, lams = [], [], [], []
    for face in coarse_faces(g):
        sup, val = snapshots(g, A, B, blocks, face)
        a, s = spectral_problem(g, A, B, kinv, face, sup, val)
        lam, cset = solve_spectral(a, s, tol, cap)
        _, low = solve_spectral(a, s, np.inf, k)       # the k lowest eigenfunctions
        X.append(face_input(kap, g, face))
        Q.append(face_label(low, a, k).T)
        nsel.append(cset.shape[1])
        lams.append(lam)
    return np.array(X), np.array(Q), np.array(nsel), np.array(lams)


__all__ = ["input_shape", "face_input", "face_label", "bf16", "param_layout", "unpack", "pack", "forward",
           "subspace_loss", "backward", "loss_and_grad", "adam_step", "ritz_select", "exact_profiles",
           "face_blocks", "fine_faces_on"]
