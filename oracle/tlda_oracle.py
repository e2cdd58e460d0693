"""FP64 oracle for the online Tensor LDA hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library; the only common module is the seeded input generator ``tlda_synth``.

Plain numpy/scipy in float64, written step by step from the paper
"Analyzing Political Text at Scale with Online Tensor LDA" (Kangaslahti et al.).
Library primitives (dense matmul, sparse CSR products, symmetric eigh, the
Hungarian assignment) serve as single steps; nothing is blocked or fused,
except in whitened_third_moment_chunked, which adds the same per-document and
per-word sums as whitened_third_moment in chunks (so that the k^3 tensor of a
corpus of millions of documents fits in memory and time) and takes the pair
term as Z^T Z - W^T diag(C) W instead of forming the V x V pair counts.

Notation: F is the B x V count matrix of a batch (CSR), f_d its rows,
L_d = sum_m f_dm, W (V x k) the whitening, m1 = W^T M1, u_m = w_m - m1
(U = W - 1 m1^T), Phi (k x K) the CP factors, c3 = (alpha0+1)(alpha0+2)/2.

Readings of the paper adopted here (where it is silent, garbled or at odds
with itself):
  A  pooled token normalisation: M1 = C/T, pair sums / S2, triple sums / S3,
     with T = sum L, S2 = sum L(L-1), S3 = sum L(L-1)(L-2).
  B  same-token corrections are kept: the third moment is taken over ordered
     triples of DISTINCT tokens (inclusion-exclusion), as in the appendix
     cumulant; ``same_token=False`` drops them (the data term of eq. vec_deriv
     on this normalisation).
  C  the alpha0 term of M3 is the one of the Theorem-1 proof:
     -alpha0(alpha0+1)/2 * sum over the 3 placements of E2 (x) M1.
  D/E whitening by the UNCENTRED M2 (rank K): W^T M2 W = I, W = U_k Lambda_k^-1/2.
     The decomposed tensor is T = M3(W,W,W), written in centred form through
     Theorem 1; its factors are the topics mu_i themselves.
  F  Phi unconstrained (no unit-norm projection); weights ride on ||phi_i||.
  G  lambda_i = ||phi_i||^3, alpha_i proportional to lambda_i^-2, sum 1.
  L  in the batch tensor, whitened M2 is replaced by I (its defining value).
  P  the fully online mode's incremental PCA is a one-pass sketch Z = P Omega
     of the pair counts (Omega: V x r Gaussian test matrix, an input), with
     the whitening rebuilt from it by the single-pass eigendecomposition of
     Halko, Martinsson and Tropp (2011, section 5.5), which also holds for
     the indefinite M2 of a small sample.
  Q  in that mode, batches go in blocks of `every`: a block's documents update
     the statistics and the whitening first, then its CP steps run (every = 1
     is the paper's per-batch order); on a change of whitening the factors
     are carried into the new basis so that the topics they encode stay put.
  R  the batched mode's loop over the data for the third moment runs from
     several initial factor matrices and keeps the one whose last epoch has
     the lowest mean loss: the unconstrained objective (reading F) has
     spurious stationary points (a collapsed component, two components on
     one topic) that a single start may end in.  The simulations' score is
     the Pearson correlation of each true topic with its learned match, under
     the one-to-one matching of largest total correlation.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.special
from scipy.optimize import linear_sum_assignment

# ----------------------------------------------------------------------------- O1 ingest


def validate_csr(indptr, indices, counts, V):
    """Raise ValueError unless (indptr, indices, counts) is a valid count CSR:
    indptr non-decreasing from indptr[0] >= 0, indices in [0, V) strictly
    ascending within each row, counts > 0 (the document-term matrix F of
    section "Computing the Centered Cumulants")."""
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    counts = np.asarray(counts, dtype=np.int64)
    if indptr.ndim != 1 or len(indptr) < 1:
        raise ValueError("indptr must have n_docs+1 entries")
    if indptr[0] < 0 or np.any(np.diff(indptr) < 0):
        raise ValueError("indptr must be non-decreasing and start >= 0")
    lo, hi = int(indptr[0]), int(indptr[-1])
    if hi > len(indices) or hi > len(counts):
        raise ValueError("indptr points past indices/counts")
    idx, cnt = indices[lo:hi], counts[lo:hi]
    if np.any(idx < 0) or np.any(idx >= V):
        raise ValueError("word index outside [0, V)")
    if np.any(cnt <= 0):
        raise ValueError("count <= 0")
    for d in range(len(indptr) - 1):
        row = indices[indptr[d]:indptr[d + 1]]
        if np.any(np.diff(row) <= 0):
            raise ValueError(f"row {d}: indices not strictly ascending")


def csr_matrix(indptr, indices, counts, V) -> sp.csr_matrix:
    """F as a float64 scipy CSR matrix (rows rebased to indptr[0])."""
    indptr = np.asarray(indptr, dtype=np.int64)
    lo, hi = int(indptr[0]), int(indptr[-1])
    return sp.csr_matrix((np.asarray(counts[lo:hi], dtype=np.float64),
                          np.asarray(indices[lo:hi], dtype=np.int64), indptr - lo),
                         shape=(len(indptr) - 1, V))


def ingest(indptr, indices, counts, V):
    """Integer statistics of a batch (reading A), all exact int64:
    L_d (row sums), C_m = sum_d f_dm, T = sum L, S2 = sum L(L-1),
    S3 = sum L(L-1)(L-2)."""
    validate_csr(indptr, indices, counts, V)
    indptr = np.asarray(indptr, dtype=np.int64)
    lo, hi = int(indptr[0]), int(indptr[-1])
    cnt = np.asarray(counts[lo:hi], dtype=np.int64)
    idx = np.asarray(indices[lo:hi], dtype=np.int64)
    B = len(indptr) - 1
    rows = np.repeat(np.arange(B), np.diff(indptr))
    L = np.zeros(B, dtype=np.int64)
    np.add.at(L, rows, cnt)
    C = np.zeros(V, dtype=np.int64)
    np.add.at(C, idx, cnt)
    return dict(L=L, C=C, T=int(L.sum()), S2=int(np.sum(L * (L - 1))),
                S3=int(np.sum(L * (L - 1) * (L - 2))))


# ----------------------------------------------------------------------------- O2/O3 moments


def first_moment(C, T):
    """M1 (eq. M1 of the appendix "Uncentered cumulants"), pooled over tokens:
    M1 = C / T (reading A)."""
    return np.asarray(C, dtype=np.float64) / float(T)


def pair_counts(indptr, indices, counts, V):
    """P = sum_d (f_d f_d^T - diag f_d): ordered pairs of distinct tokens per
    word pair (the bracket of the appendix M2), exact int64, V x V."""
    F = csr_matrix(indptr, indices, counts, V)
    P = (F.T @ F).toarray()
    C = np.asarray(F.sum(axis=0)).ravel()
    P = np.rint(P).astype(np.int64)
    P[np.diag_indices(V)] -= np.rint(C).astype(np.int64)
    return P


def second_moment(P, S2, M1, alpha0):
    """Uncentred M2 = (alpha0+1) E2 - alpha0 M1 M1^T with E2 = P / S2
    (appendix "Uncentered cumulants", eq. M2; pooled normalisation, reading A)."""
    return (alpha0 + 1.0) * (P.astype(np.float64) / float(S2)) - alpha0 * np.outer(M1, M1)


# ----------------------------------------------------------------------------- O4 whitening


def whitening(M2, k):
    """Top-k eigenpairs of M2 and W = U_k Lambda_k^-1/2, so that W^T M2 W = I
    (section "Online Decomposition of the Second Moment", readings D/E).
    Eigenpairs in descending order; each eigenvector's sign makes its
    largest-magnitude entry positive (lowest index on ties).
    Returns (W, U_k, lambda_k)."""
    M2 = 0.5 * (M2 + M2.T)
    lam, vec = np.linalg.eigh(M2)
    order = np.argsort(-lam, kind="stable")[:k]
    lam, vec = lam[order], vec[:, order]
    if not (lam[-1] > 1e-12 * lam[0]):
        raise ValueError("M2 has fewer than k positive eigenvalues")
    for j in range(k):
        i = int(np.argmax(np.abs(vec[:, j])))
        if vec[i, j] < 0:
            vec[:, j] = -vec[:, j]
    W = vec / np.sqrt(lam)[None, :]
    return W, vec, lam


# ----------------------------------------------------------------------------- O5 explicit M3


def sym3(a, b, c):
    """a (x) b (x) c for vectors."""
    return np.einsum("i,j,l->ijl", a, b, c)


def perm3(Mat, v):
    """Sum over the three placements of a matrix and a vector:
    Mat_ij v_l + Mat_il v_j + v_i Mat_jl."""
    return (np.einsum("ij,l->ijl", Mat, v) + np.einsum("il,j->ijl", Mat, v)
            + np.einsum("i,jl->ijl", v, Mat))


def whitened_third_moment(indptr, indices, counts, V, W, M1, alpha0):
    """T_full = M3(W, W, W) for the uncentred third cumulant of the appendix
    ("Uncentered cumulants", eq. M3) with the alpha0 term of the Theorem-1 proof
    (reading C) and pooled normalisation (reading A):
      T_full = c3 E3w - alpha0(alpha0+1)/2 * perm3(E2w, m1) + alpha0^2 m1^(x)3,
      E3w = (1/S3) sum_d [z_d^(x)3 - perm3(A_d, z_d) + 2 sum_m f_dm w_m^(x)3],
      z_d = W^T f_d, A_d = sum_m f_dm w_m w_m^T, E2w = W^T (P/S2) W, m1 = W^T M1.
    Explicit k^3 tensor: small k only."""
    st = ingest(indptr, indices, counts, V)
    F = csr_matrix(indptr, indices, counts, V)
    Z = F @ W                                   # z_d rows
    C = st["C"].astype(np.float64)
    Hm = F.T @ Z                                # h_m = sum_d f_dm z_d
    zzz = np.einsum("di,dj,dl->ijl", Z, Z, Z)
    # sum_d perm3(A_d, z_d) = sum_m [w_m w_m^T (x) h_m + ...] over the placements
    awz = (np.einsum("mi,mj,ml->ijl", W, W, Hm) + np.einsum("mi,ml,mj->ijl", W, W, Hm)
           + np.einsum("mj,ml,mi->ijl", W, W, Hm))
    www = np.einsum("m,mi,mj,ml->ijl", C, W, W, W)
    E3w = (zzz - awz + 2.0 * www) / float(st["S3"])
    P = pair_counts(indptr, indices, counts, V)
    E2w = W.T @ (P.astype(np.float64) / float(st["S2"])) @ W
    m1 = W.T @ M1
    c3 = (alpha0 + 1.0) * (alpha0 + 2.0) / 2.0
    return (c3 * E3w - alpha0 * (alpha0 + 1.0) / 2.0 * perm3(E2w, m1)
            + alpha0 ** 2 * sym3(m1, m1, m1))


# ----------------------------------------------------------------------------- O6 batch tensor


def whitened_third_moment_chunked(indptr, indices, counts, V, W, M1, alpha0, chunk=2048):
    """The tensor of whitened_third_moment (same definition, readings A and C),
    for corpora too large for its einsums: the sums over documents and over
    words are added chunk by chunk, each chunk's sum of outer products taken
    as one matrix product (Z_c^T times the rows z_d (x) z_d of the chunk), and
    W^T P W = sum_d (z_d z_d^T) - W^T diag(C) W, the pair counts
    P = sum_d (f_d f_d^T - diag f_d) mapped through W without forming P."""
    st = ingest(indptr, indices, counts, V)
    F = csr_matrix(indptr, indices, counts, V)
    k = W.shape[1]
    C = st["C"].astype(np.float64)
    zzz = np.zeros((k, k * k))
    ZtZ = np.zeros((k, k))
    Hm = np.zeros((V, k))
    n = F.shape[0]
    for d0 in range(0, n, chunk):
        Fc = F[d0:d0 + chunk]
        Zc = np.asarray(Fc @ W)                                  # z_d rows
        zzz += Zc.T @ (Zc[:, :, None] * Zc[:, None, :]).reshape(-1, k * k)
        ZtZ += Zc.T @ Zc
        Hm += np.asarray(Fc.T @ Zc)                              # h_m = sum_d f_dm z_d
    zzz = zzz.reshape(k, k, k)
    wwh = np.zeros((k * k, k))
    www = np.zeros((k * k, k))
    for m0 in range(0, V, chunk):
        Wc = W[m0:m0 + chunk]
        ww = (Wc[:, :, None] * Wc[:, None, :]).reshape(-1, k * k)  # rows w_m (x) w_m
        wwh += ww.T @ Hm[m0:m0 + chunk]
        www += ww.T @ (C[m0:m0 + chunk, None] * Wc)
    wwh = wwh.reshape(k, k, k)                                   # sum_m w_m (x) w_m (x) h_m
    awz = wwh + wwh.transpose(0, 2, 1) + wwh.transpose(2, 0, 1)  # the three placements of h_m
    E3w = (zzz - awz + 2.0 * www.reshape(k, k, k)) / float(st["S3"])
    E2w = (ZtZ - W.T @ (C[:, None] * W)) / float(st["S2"])
    m1 = W.T @ M1
    c3 = (alpha0 + 1.0) * (alpha0 + 2.0) / 2.0
    return (c3 * E3w - alpha0 * (alpha0 + 1.0) / 2.0 * perm3(E2w, m1)
            + alpha0 ** 2 * sym3(m1, m1, m1))


def centred_triples(indptr, indices, counts, V, W, m1):
    """(1/S3) sum_d sum over ordered triples of distinct tokens of
    u_t1 (x) u_t2 (x) u_t3, u_m = w_m - m1, by inclusion-exclusion:
      sum_d [x_d^(x)3 - perm3(A'_d, x_d) + 2 sum_m f_dm u_m^(x)3],
    x_d = sum_m f_dm u_m, A'_d = sum_m f_dm u_m u_m^T  (reading B).
    Returns (C3hat, S3)."""
    st = ingest(indptr, indices, counts, V)
    F = csr_matrix(indptr, indices, counts, V)
    U = W - m1[None, :]
    X = F @ U
    Hm = F.T @ X
    C = st["C"].astype(np.float64)
    xxx = np.einsum("di,dj,dl->ijl", X, X, X)
    aux = (np.einsum("mi,mj,ml->ijl", U, U, Hm) + np.einsum("mi,ml,mj->ijl", U, U, Hm)
           + np.einsum("mj,ml,mi->ijl", U, U, Hm))
    uuu = np.einsum("m,mi,mj,ml->ijl", C, U, U, U)
    S3 = st["S3"]
    if S3 == 0:
        return np.zeros((W.shape[1],) * 3), 0
    return (xxx - aux + 2.0 * uuu) / float(S3), S3


def batch_tensor(indptr, indices, counts, V, W, m1, alpha0):
    """Whitened uncentred M3 of a batch in centred form (Theorem 1 with
    W^T M2 W = I, readings E and L):
        T_B = c3 C3hat + perm3(I, m1) - 2 m1^(x)3."""
    C3, S3 = centred_triples(indptr, indices, counts, V, W, m1)
    k = W.shape[1]
    c3 = (alpha0 + 1.0) * (alpha0 + 2.0) / 2.0
    return c3 * C3 + perm3(np.eye(k), m1) - 2.0 * sym3(m1, m1, m1)


# ----------------------------------------------------------------------------- O8 CP objective


def cp_loss_explicit(Phi, T, theta):
    """Loss of eq. vec_pb with unconstrained factors (reading F):
    (1+theta)/2 ||sum_i phi_i^(x)3||^2 - <sum_i phi_i^(x)3, T>."""
    G = Phi.T @ Phi
    return (1.0 + theta) / 2.0 * float(np.sum(G ** 3)) - float(
        np.einsum("ijl,ia,ja,la->", T, Phi, Phi, Phi))


def cp_grad_explicit(Phi, T, theta):
    """Gradient of cp_loss_explicit (eq. vec_deriv with T in place of the
    sample third moment): 3(1+theta) Phi (Phi^T Phi * Phi^T Phi)
    - 3 [T(I, phi_i, phi_i)]_i."""
    G = Phi.T @ Phi
    return 3.0 * (1.0 + theta) * Phi @ (G * G) - 3.0 * np.einsum("ijl,ja,la->ia", T, Phi, Phi)


def cp_grad_implicit(indptr, indices, counts, V, W, m1, Phi, alpha0, theta, same_token=True):
    """The CP gradient of one minibatch without forming any k^3 tensor, in the
    order of the hot path:
      a1  L_d, S3 (ingest)
      a2  X = F W - L m1^T                       (= F U)
      a3  Y = X Phi
      a4  Q = U Phi,  R = F (Q*Q)
      a5  G1 = X^T (Y*Y - R)
      a6  H = F^T Y,  G2 = U^T [Q * (2 c*Q - 2 H)],  c_m = sum_d f_dm
      a7  G3_i = 2 phi_i (m1.phi_i) + m1 ||phi_i||^2 - 2 m1 (m1.phi_i)^2
      a8  P = Phi (Phi^T Phi * Phi^T Phi)
      a9  grad = 3(1+theta) P - 3 [c3/S3 (G1 + G2) + G3]
    This equals cp_grad_explicit(Phi, batch_tensor(...)) exactly in exact
    arithmetic (eq. vec_deriv's data term with the same-token terms of
    reading B).  With same_token=False, R and G2 are dropped.
    S3 == 0 (no document with three tokens): the batch carries no triple, so
    the step is defined as a no-op (grad = 0, loss = 0).
    Returns a dict with every intermediate."""
    st = ingest(indptr, indices, counts, V)
    k, K = Phi.shape
    out = dict(S3=st["S3"], L=st["L"], C=st["C"])
    if st["S3"] == 0:
        z = np.zeros((k, K))
        out.update(grad=z, G_data=z, G1=z, G2=z, G3=z, P=z, loss=0.0)
        return out
    F = csr_matrix(indptr, indices, counts, V)
    U = W - m1[None, :]
    X = F @ W - st["L"][:, None].astype(np.float64) * m1[None, :]        # a2
    Y = X @ Phi                                                           # a3
    Q = U @ Phi                                                           # a4
    R = F @ (Q * Q)
    if not same_token:
        R = np.zeros_like(R)
    G1 = X.T @ (Y * Y - R)                                                # a5
    if same_token:                                                        # a6
        H = F.T @ Y
        c = st["C"].astype(np.float64)[:, None]
        G2 = U.T @ (Q * (2.0 * c * Q - 2.0 * H))
    else:
        G2 = np.zeros_like(G1)
    a = m1 @ Phi                                                          # a7
    nrm2 = np.sum(Phi * Phi, axis=0)
    G3 = 2.0 * Phi * a[None, :] + np.outer(m1, nrm2) - 2.0 * np.outer(m1, a * a)
    G = Phi.T @ Phi                                                       # a8
    Pm = Phi @ (G * G)
    c3 = (alpha0 + 1.0) * (alpha0 + 2.0) / 2.0
    G_data = c3 / float(st["S3"]) * (G1 + G2) + G3
    grad = 3.0 * (1.0 + theta) * Pm - 3.0 * G_data                        # a9
    # loss: (1+theta)/2 sum (Phi^T Phi)^3 - sum_i T_B(phi_i, phi_i, phi_i)
    cube = np.sum(Y ** 3 - 3.0 * Y * R, axis=0)
    if same_token:
        cube = cube + 2.0 * np.sum(st["C"].astype(np.float64)[:, None] * Q ** 3, axis=0)
    tb = c3 / float(st["S3"]) * cube + 3.0 * a * nrm2 - 2.0 * a ** 3
    loss = (1.0 + theta) / 2.0 * float(np.sum(G ** 3)) - float(np.sum(tb))
    out.update(X=X, Y=Y, Q=Q, R=R, G1=G1, G2=G2, G3=G3, P=Pm, G_data=G_data, grad=grad,
               loss=loss)
    return out


def cp_step(indptr, indices, counts, V, W, m1, Phi, lr, alpha0, theta, same_token=True):
    """One stochastic tensor gradient step (section "Online Learning of the
    Third Moment"): Phi_{t+1} = Phi_t - beta * dL/dPhi."""
    g = cp_grad_implicit(indptr, indices, counts, V, W, m1, Phi, alpha0, theta, same_token)
    return Phi - lr * g["grad"], g


# ----------------------------------------------------------------------------- O7 power method


def tensor_power_method(T, K, n_restarts=30, n_iters=100, seed=0):
    """Robust tensor power method with deflation (Anandkumar, Ge, Hsu, Kakade,
    Telgarsky 2014, "Tensor decompositions for learning latent variable
    models", Algorithm 1), the spectral decomposition the paper builds on.
    Returns (lambda (K,), V (k x K)) with lambda_i > 0."""
    rng = np.random.default_rng(seed)
    T = T.copy()
    k = T.shape[0]
    lams, vecs = [], []
    for _ in range(K):
        best, best_val = None, -np.inf
        for _ in range(n_restarts):
            th = rng.standard_normal(k)
            th /= np.linalg.norm(th)
            for _ in range(n_iters):
                nxt = np.einsum("ijl,j,l->i", T, th, th)
                nn = np.linalg.norm(nxt)
                if nn == 0.0:
                    break
                th = nxt / nn
            val = float(np.einsum("ijl,i,j,l->", T, th, th, th))
            if val > best_val:
                best, best_val = th, val
        th = best
        for _ in range(n_iters):
            nxt = np.einsum("ijl,j,l->i", T, th, th)
            th = nxt / np.linalg.norm(nxt)
        lam = float(np.einsum("ijl,i,j,l->", T, th, th, th))
        if lam < 0:
            lam, th = -lam, -th
        lams.append(lam)
        vecs.append(th)
        T = T - lam * sym3(th, th, th)
    return np.array(lams), np.stack(vecs, axis=1)


# ----------------------------------------------------------------------------- O9 recovery


def pinv_transpose(W):
    """(W^T)^dagger = W (W^T W)^-1 for full-column-rank W (section
    "Recovering the Topic Model Parameters")."""
    return W @ np.linalg.inv(W.T @ W)


def unwhiten_power(lams, Vecs, W):
    """Topics from eigenpairs of T = sum_i lambda_i v_i^(x)3:
    mu_i = lambda_i (W^T)^dagger v_i, weights h_i = lambda_i^-2 (normalised)."""
    mu = pinv_transpose(W) @ (Vecs * lams[None, :])
    h = lams ** -2.0
    return mu, h / h.sum()


def unwhiten_cp(Phi, W):
    """Topics from CP factors (reading G): lambda_i = ||phi_i||^3,
    v_i = phi_i/||phi_i||, so mu_i = ||phi_i||^2 (W^T)^dagger phi_i and
    alpha_i proportional to ||phi_i||^-6 (sum 1).  Returns raw mu (V x K,
    unclipped) and alpha."""
    n = np.linalg.norm(Phi, axis=0)
    mu = pinv_transpose(W) @ (Phi * (n ** 2)[None, :])
    a = n ** -6.0
    return mu, a / a.sum()


def clip_normalise(mu):
    """Clip topic-word estimates at 0 and renormalise each topic to sum 1.
    Returns (mu, clipped negative mass per topic)."""
    neg = -np.minimum(mu, 0.0).sum(axis=0)
    m = np.maximum(mu, 0.0)
    s = m.sum(axis=0)
    s[s == 0] = 1.0
    return m / s[None, :], neg


# ----------------------------------------------------------------------------- O10 scoring


def match_topics(mu_est, mu_true):
    """Hungarian assignment on per-topic l1 distance. mu_est: V x K (columns
    topics), mu_true: K x V.  Returns (perm, l1 per matched topic, correlation
    per matched topic), est column perm[i] matched to true topic i."""
    K = mu_true.shape[0]
    D = np.abs(mu_true[:, :, None] - mu_est[None, :, :]).sum(axis=1)   # K x K
    r, c = linear_sum_assignment(D)
    perm = np.empty(K, dtype=np.int64)
    perm[r] = c
    l1 = D[np.arange(K), perm]
    corr = np.array([np.corrcoef(mu_true[i], mu_est[:, perm[i]])[0, 1] for i in range(K)])
    return perm, l1, corr


# ----------------------------------------------------------------------------- population


def population_moments(mu, h):
    """Closed forms of the moments (section "Computing the Centered
    Cumulants" factorisation and Theorem 1): with h_i = alpha_i/alpha0,
    M1 = sum h_i mu_i, M2 = sum h_i mu_i mu_i^T, M3 = sum h_i mu_i^(x)3.
    mu: K x V.  M3 is V^3: small V only (pass want_m3=False otherwise)."""
    M1 = h @ mu
    M2 = (mu.T * h[None, :]) @ mu
    return M1, M2


def population_m3(mu, h):
    return np.einsum("k,ki,kj,kl->ijl", h, mu, mu, mu)


def population_whitening(mu, h):
    """W with W^T M2 W = I for the rank-K population M2 = A A^T,
    A = mu^T diag(sqrt h), through the K x K Gram matrix: A^T A = E S E^T,
    U = A E S^-1/2, W = U S^-1/2 (so no V x V matrix is formed).
    Returns (W, m1 = W^T M1)."""
    A = mu.T * np.sqrt(h)[None, :]
    S, E = np.linalg.eigh(A.T @ A)
    order = np.argsort(-S)
    S, E = S[order], E[:, order]
    W = A @ E / S[None, :]
    M1 = h @ mu
    return W, W.T @ M1


def population_tensor(mu, h, W):
    """T = M3(W, W, W) = sum_i h_i (W^T mu_i)^(x)3 (whitened, orthogonal:
    lambda_i = h_i^-1/2)."""
    Wm = W.T @ mu.T
    return np.einsum("k,ik,jk,lk->ijl", h, Wm, Wm, Wm)


def population_factors(mu, h, W):
    """Stationary CP factors of the population tensor at theta = 0:
    phi_i = h_i^(1/3) W^T mu_i (so ||phi_i|| = h_i^-1/6, lambda_i = h_i^-1/2)."""
    return (W.T @ mu.T) * (h ** (1.0 / 3.0))[None, :]


# ----------------------------------------------------------------------------- online mode


def sketch_accumulate(indptr, indices, counts, V, Omega):
    """A batch's part of the one-pass sketch Z = P Omega of the pair counts
    P = sum_d (f_d f_d^T - diag f_d) (the numerator of O3; reading P):
    row m is sum_d f_dm (f_d^T Omega - Omega_m)."""
    F = csr_matrix(indptr, indices, counts, V)
    S = F @ Omega                                # B x r rows f_d^T Omega
    c = np.asarray(F.sum(axis=0)).ravel()        # c_m = sum_d f_dm
    return F.T @ S - c[:, None] * Omega


def sketch_eigenpairs(Y, Omega, k):
    """Top-k eigenpairs of a symmetric matrix A from Y = A Omega alone (the
    single-pass eigenvalue decomposition of Halko, Martinsson and Tropp 2011,
    section 5.5): Q R = Y (thin QR), B solves B (Q^T Omega) = Q^T Y in the
    least-squares sense, B is symmetrised, B = E Lambda E^T, U = Q E.  Exact
    when range(A) lies in range(Y) (rank A <= r, or r = V).  Pairs in
    descending order, each vector's largest-magnitude entry made positive
    (reading J).  Returns (U_k, Lambda_k)."""
    Q, R = np.linalg.qr(Y)
    C2 = Q.T @ Omega
    B = np.linalg.lstsq(C2.T, R.T, rcond=None)[0].T
    B = 0.5 * (B + B.T)
    lam, E = np.linalg.eigh(B)
    order = np.argsort(-lam, kind="stable")[:k]
    lam, U = lam[order], Q @ E[:, order]
    for j in range(k):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
    return U, lam


def sketch_whitening(Z, C, T, S2, Omega, alpha0, k):
    """The whitening of the online mode (reading P): with M1 = C/T, the sketch
    of M2 = (alpha0+1) P/S2 - alpha0 M1 M1^T (O3) is
    Y = (alpha0+1)/S2 Z - alpha0 M1 (M1^T Omega); its eigenpairs
    (``sketch_eigenpairs``) give W = U_k Lambda_k^-1/2.
    Returns (W, m1 = W^T M1, Lambda_k)."""
    M1 = np.asarray(C, dtype=np.float64) / float(T)
    Y = (alpha0 + 1.0) / float(S2) * Z - alpha0 * np.outer(M1, M1 @ Omega)
    U, lam = sketch_eigenpairs(Y, Omega, k)
    if not (lam[-1] > 1e-12 * lam[0]):
        raise ValueError("the sketched M2 has fewer than k positive eigenvalues")
    W = U / np.sqrt(lam)[None, :]
    return W, W.T @ M1, lam


def rotate_factors(Phi, W_old, W_new):
    """CP factors carried into a new whitened basis (reading Q).  The topics
    they encode, mu_i proportional to (W^T)^dagger phi_i (section "Recovering
    the Topic Model Parameters"), stay put:
    phi_i' = W_new^T (W_old^T)^dagger phi_i."""
    return W_new.T @ (pinv_transpose(W_old) @ Phi)


def online_pass(indptr, indices, counts, V, offsets, Omega, every, alpha0, theta, lr, Phi, k,
                same_token=True, state=None):
    """One fully online pass (section "Fully Online Implementation", readings
    P and Q): batch b is documents [offsets[b], offsets[b+1]); the batches go
    in blocks of `every`.  For each block its documents first update the token
    statistics (C, T, S2) and the sketch Z, the whitening is rebuilt from the
    sketch (``sketch_whitening``) and Phi carried into it, then the block's
    CP steps run in order.
    `state` (C, T, S2, Z, W, m1) carries over between calls.  Returns
    (Phi, state, losses)."""
    indptr = np.asarray(indptr, dtype=np.int64)
    if state is None:
        state = dict(C=np.zeros(V, dtype=np.int64), T=0, S2=0, Z=np.zeros_like(Omega), W=None, m1=None)
    Phi = np.array(Phi, dtype=np.float64)
    losses = []
    nb = len(offsets) - 1
    for b0 in range(0, nb, every):
        b1 = min(nb, b0 + every)
        d0, d1 = int(offsets[b0]), int(offsets[b1])
        rows = indptr[d0:d1 + 1]
        st = ingest(rows, indices, counts, V)
        state["C"] = state["C"] + st["C"]
        state["T"] += st["T"]
        state["S2"] += st["S2"]
        state["Z"] = state["Z"] + sketch_accumulate(rows, indices, counts, V, Omega)
        W, m1, _ = sketch_whitening(state["Z"], state["C"], state["T"], state["S2"], Omega, alpha0, k)
        if state["W"] is not None:
            Phi = rotate_factors(Phi, state["W"], W)
        state["W"], state["m1"] = W, m1
        for b in range(b0, b1):
            r = indptr[int(offsets[b]):int(offsets[b + 1]) + 1]
            Phi, g = cp_step(r, indices, counts, V, W, m1, Phi, lr, alpha0, theta, same_token)
            losses.append(g["loss"])
    return Phi, state, np.array(losses)


# ----------------------------------------------------------------------------- batched mode


def batched_fit(indptr, indices, counts, V, offsets, epochs, alpha0, theta, lr, Phi_starts, k,
                same_token=True):
    """The batched mode (section "Batched Implementation Enables Arbitrary
    Scaling"; reading R): the moments and the whitening from the whole corpus
    (O1-O4), then `epochs` passes of CP steps over the batches
    [offsets[b], offsets[b+1]) from each initial factor matrix; the start
    whose last epoch has the lowest mean loss is kept (NaN never wins).
    Returns (kept Phi, W, m1, mean last-epoch loss per start, final Phi per start)."""
    indptr = np.asarray(indptr, dtype=np.int64)
    st = ingest(indptr, indices, counts, V)
    M1 = first_moment(st["C"], st["T"])
    M2 = second_moment(pair_counts(indptr, indices, counts, V), st["S2"], M1, alpha0)
    W, _, _ = whitening(M2, k)
    m1 = W.T @ M1
    finals, means = [], []
    for P0 in Phi_starts:
        P = np.array(P0, dtype=np.float64)
        for _ in range(epochs):
            losses = []
            for b in range(len(offsets) - 1):
                r = indptr[int(offsets[b]):int(offsets[b + 1]) + 1]
                P, g = cp_step(r, indices, counts, V, W, m1, P, lr, alpha0, theta, same_token)
                losses.append(g["loss"])
        means.append(float(np.mean(losses)))
        finals.append(P)
    means = np.array(means)
    ok = np.flatnonzero(np.isfinite(means))
    best = int(ok[np.argmin(means[ok])]) if len(ok) else 0
    return finals[best], W, m1, means, finals


def topic_correlation(mu_est, mu_true):
    """Recovery score of the simulations (section "Parameter Recovery and
    Comparison to Previous TLDA Methods"; reading R): the Pearson correlation
    of each true topic-word distribution (row i of mu_true, K x V) with a
    learned one (column j of mu_est, V x K), under the one-to-one matching
    that maximises the total correlation (Hungarian assignment).  A constant
    column correlates 0 with everything.  Returns (perm, correlation per true
    topic), learned column perm[i] matched to true topic i."""
    K = mu_true.shape[0]
    Cm = np.zeros((K, K))
    for i in range(K):
        a = mu_true[i] - mu_true[i].mean()
        for j in range(K):
            b = mu_est[:, j] - mu_est[:, j].mean()
            den = np.linalg.norm(a) * np.linalg.norm(b)
            Cm[i, j] = float(a @ b) / den if den > 0 else 0.0
    r, c = linear_sum_assignment(-Cm)
    perm = np.empty(K, dtype=np.int64)
    perm[r] = c
    return perm, Cm[np.arange(K), perm]


# ----------------------------------------------------------------------------- document-topic VI


def doc_topics(indptr, indices, counts, V, mu, alpha, n_iter):
    """Document-level parameters from the recovered topics by standard
    variational inference (section "Input and Output": topic-word matrix and
    weights fed to VI), the per-document E-step of Blei, Ng and Jordan (2003,
    section 5.2) with the topics fixed.  mu: V x K (column k = topic k),
    alpha: the K Dirichlet parameters (alpha0 times the learned weights).
    Per document, gamma = alpha + L/K, then n_iter rounds of
        phi_jk proportional to mu_{m_j k} exp(digamma(gamma_k))  (over k),
        gamma_k = alpha_k + sum_j f_j phi_jk;
    a word whose mu row is all zero gets phi = 0.  Returns (theta = gamma /
    sum gamma, gamma), both B x K."""
    indptr = np.asarray(indptr, dtype=np.int64)
    mu = np.asarray(mu, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    B, K = len(indptr) - 1, mu.shape[1]
    gamma = np.zeros((B, K))
    for d in range(B):
        lo, hi = int(indptr[d]), int(indptr[d + 1])
        m = np.asarray(indices[lo:hi], dtype=np.int64)
        f = np.asarray(counts[lo:hi], dtype=np.float64)
        g = alpha + f.sum() / K
        rows = mu[m]                                          # nnz x K
        for _ in range(n_iter):
            _, g = vi_update(f, rows, alpha, g)
        gamma[d] = g
    return gamma / gamma.sum(axis=1, keepdims=True), gamma


def vi_update(f, rows, alpha, gamma):
    """One round of the E-step for one document (counts f of its words, their
    topic rows nnz x K): phi_jk proportional to rows_jk exp(digamma(gamma_k)),
    then gamma' = alpha + f^T phi.  Returns (phi, gamma')."""
    p = rows * np.exp(scipy.special.digamma(gamma))[None, :]
    s = p.sum(axis=1, keepdims=True)
    phi = np.divide(p, s, out=np.zeros_like(p), where=s > 0)
    return phi, alpha + f @ phi


def doc_elbo(f, rows, alpha, gamma, phi):
    """The per-document evidence lower bound of LDA with fixed topics (Blei,
    Ng and Jordan 2003, appendix A.3), for counts f of words with topic rows
    `rows` (nnz x K), variational Dirichlet gamma and multinomials phi
    (nnz x K, one per distinct word, shared by its f tokens)."""
    dg = scipy.special.digamma(gamma) - scipy.special.digamma(gamma.sum())
    gl = scipy.special.gammaln
    e_logtheta = (scipy.special.gammaln(alpha.sum()) - gl(alpha).sum() + ((alpha - 1.0) * dg).sum())
    with np.errstate(divide="ignore", invalid="ignore"):
        logrows = np.where(rows > 0, np.log(np.where(rows > 0, rows, 1.0)), 0.0)
        logphi = np.where(phi > 0, np.log(np.where(phi > 0, phi, 1.0)), 0.0)
    e_z = (f[:, None] * phi * dg[None, :]).sum()
    e_w = (f[:, None] * phi * logrows).sum()
    h_theta = -(gl(gamma.sum()) - gl(gamma).sum() + ((gamma - 1.0) * dg).sum())
    h_z = -(f[:, None] * phi * logphi).sum()
    return e_logtheta + e_z + e_w + h_theta + h_z
