"""CPU oracle for the filtered incremental scaling-and-squaring method
(Wu, Zhang, Zhu, Hu, "High-performance computation of large sparse matrix
exponential", arXiv 2110.04493).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path; it is a plain, slow restatement of the paper written with
numpy / scipy.sparse in float64, following Algorithm 4.2 step by step.

Readings of the paper taken here (the paper is silent or ambiguous on them):

* Norm: the Frobenius norm everywhere (Sec. 5 states it is used in all
  experiments).
* (M, N), Eq. (4.20): N in [N0, N0 + 50], N0 = max(ceil(log2 ||H||), 0);
  m(N) is the smallest M >= 1 meeting the error bound; the pair minimising
  M 2^N wins, ties going to the smaller M + N, then the smaller N.
  ||H|| = 0 gives M = N = 0 and e^H = I.
* Normality (Algorithm 4.2 step 2): H == H^T or H == -H^T exactly counts as
  normal; otherwise H is normal iff ||H H^T - H^T H||_F <= 64 u ||H||_F^2.
* Algorithm 4.1: the sentinel b_0 = 1 is read as "run the first pass with
  eps_f = eps_g unconditionally", so the guarantee
  ||A - A_tilde|| <= eps_g (1 + e_r) holds for every eps_g; entries with
  |v| == eps_f are dropped (only |v| > eps_f is kept); exact zeros are
  always dropped; e_r defaults to 0.1; the loop is capped (ENOCONV).
* Taylor phase (Algorithm 4.2 step 3, Eq. (4.11)): S_1 = H_0 is not
  filtered; each S~_i is the product S^_{i-1} H_0 with every entry divided
  by i; the loop stops once a filtered term is empty (all later terms are
  then zero).  The threshold eps_g^(0) = a r_0 / (M e^{2 ||H_0||}) bounds
  ||E_j|| directly, as derived in Eq. (4.14) ("absolute").
* Squaring (Algorithm 4.2 step 4, Eq. (4.15)): T~_i = 2 T^_{i-1} + T^_{i-1}^2
  (the printed step writes T^_i on the right; Eq. (4.15) fixes the index);
  r_i = 2^i r_0 (Sec. 4.1 drops r^2).  The dropped part must satisfy
  ||B_i|| <= a r_i ||F_i|| (Sec. 4.2, "relative"); ||F_i||_F is taken as
  ||I + T~_i||_F.  The printed eps_g^(i) = a r_i without the ||F_i|| factor
  ("absolute") is available as an option.  The relative reading is the
  default because it reproduces Table 3.
* e^H = I + T^_N, the diagonal inserted where T^_N has no stored entry.
* Complex H (the method is stated for C^{n x n}): |v| is the modulus, the sums of
  Algorithm 4.1 and the Frobenius norms add |v|^2 = re^2 + im^2, and the normality
  test uses the conjugate transpose.  Real input takes exactly the real path.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np
import scipy.sparse as sp

U_ROUNDOFF = 2.0 ** -53


class OracleError(RuntimeError):
    pass


# --------------------------------------------------------------------------
# Norms and scalar bounds
# --------------------------------------------------------------------------

def abs2(v) -> np.ndarray:
    """|v|^2 of real or complex values (re^2 + im^2 for complex)."""
    v = np.asarray(v)
    if np.iscomplexobj(v):
        return v.real.astype(np.float64) ** 2 + v.imag.astype(np.float64) ** 2
    return np.asarray(v, dtype=np.float64) ** 2


def fro_norm(A) -> float:
    """Frobenius norm sqrt(sum |a_ij|^2) over the stored entries (Sec. 5)."""
    v = A.data if sp.issparse(A) else np.asarray(A).ravel()
    return math.sqrt(math.fsum(abs2(v).tolist())) if len(v) < 200000 else float(np.sqrt(np.sum(abs2(v))))


def rho(M: int, x: float) -> float:
    """Relative error bound of the degree-M Taylor approximant, Eq. (4.5):

    ||F_0^{-1} R_0|| <= (1/M!) sum_{k>=0} x^{M+1+k} / (k! (M+1+k)),  x = ||H 2^-N||,
    the series form of (-1)^{M+1} gamma(M+1, -x) / M!.
    """
    if x == 0.0:
        return 0.0
    c = 1.0  # x^{M+1+k} / (M! k!) built up term by term
    for j in range(1, M + 2):
        c *= x / j if j <= M else x
    # after the loop c = x^{M+1} / M!
    total = 0.0
    k = 0
    while True:
        term = c / (M + 1 + k)
        total += term
        if term <= 1e-18 * total or c == 0.0:
            break
        k += 1
        c *= x / k
        if k > 10000:
            break
    return total


def scale_pow2(v, e: int) -> np.ndarray:
    """v 2^e, exact (real or complex values)."""
    v = np.asarray(v)
    if np.iscomplexobj(v):
        return np.ldexp(v.real, e) + 1j * np.ldexp(v.imag, e)
    return np.ldexp(v, e)


def div_real(v, d) -> np.ndarray:
    """v / d for a real d, each part divided once (for complex v numpy's complex division would
    round differently)."""
    v = np.asarray(v)
    if np.iscomplexobj(v):
        return v.real / d + 1j * (v.imag / d)
    return v / d


def ceil_log2(x: float) -> int:
    """Exact ceil(log2 x) for x > 0."""
    m, e = math.frexp(x)  # x = m 2^e, 0.5 <= m < 1
    return e - 1 if m == 0.5 else e


def choose_MN(normH: float, eps_tol: float, n_extra: int = 50, m_cap: int = 1000) -> Tuple[int, int]:
    """Scaling N and Taylor degree M by the enumeration of Eq. (4.20)."""
    if normH == 0.0:
        return 0, 0
    N0 = max(ceil_log2(normH), 0)
    best = None
    for N in range(N0, N0 + n_extra + 1):
        x = math.ldexp(normH, -N)
        M = 1
        while math.ldexp(rho(M, x), N) > eps_tol:
            M += 1
            if M > m_cap:
                break
        if M > m_cap:
            continue
        key = (M * 2 ** N, M + N, N)
        if best is None or key < best[0]:
            best = (key, M, N)
    if best is None:
        raise OracleError("no feasible (M, N)")
    return best[1], best[2]


def is_normal(H: sp.csr_matrix) -> bool:
    """Normality test (reading of Algorithm 4.2 step 2, see module docstring); H^T is the
    conjugate transpose for complex H (normal: H H^* = H^* H)."""
    Ht = H.conj().T.tocsr()
    if (H != Ht).nnz == 0 or (H + Ht).count_nonzero() == 0:
        return True
    C = (H @ Ht) - (Ht @ H)
    return fro_norm(C) <= 64.0 * U_ROUNDOFF * fro_norm(H) ** 2


# --------------------------------------------------------------------------
# Algorithm 4.1
# --------------------------------------------------------------------------

@dataclasses.dataclass
class FilterInfo:
    eps_g: float
    t: float          # final eps_f: entries with |v| <= t are dropped
    iters: int
    b: float          # F-norm of the dropped part
    nnz_in: int
    nnz_out: int


def alg41_threshold(vals: np.ndarray, eps_g: float, e_r: float, max_iter: int = 100) -> Tuple[float, int, float]:
    """Algorithm 4.1 on the stored values of a matrix.

    Returns (eps_f, iterations, b): the entries with |v| > eps_f are kept, the
    rest (whose F-norm is b <= eps_g (1 + e_r)) are dropped.
    """
    vals = np.asarray(vals)
    mag = np.asarray(np.abs(vals), dtype=np.float64)  # |v|: the modulus for complex values
    sq = abs2(vals)                                   # |v|^2 (re^2 + im^2 for complex)
    m = 1.0
    b = math.inf  # the first pass always runs (reading of the b_0 sentinel)
    n = 0
    eps_f = eps_g
    while b > eps_g * (1.0 + e_r):
        if n >= max_iter:
            raise OracleError("Algorithm 4.1 did not converge")
        eps_f = eps_g / m
        keep = mag <= eps_f                    # b_n(p) = 0 for |b_n| > eps_f
        mag, sq = mag[keep], sq[keep]
        b = float(np.sqrt(np.sum(sq)))
        m = b / eps_f
        n += 1
    return eps_f, n, b


def filter_csr(A: sp.csr_matrix, eps_g: float, e_r: float, max_iter: int = 100) -> Tuple[sp.csr_matrix, FilterInfo]:
    """A_tilde = A - b_n of Algorithm 4.1: keep the stored entries with |v| > eps_f."""
    t, iters, b = alg41_threshold(A.data, eps_g, e_r, max_iter)
    keep = np.abs(A.data) > t
    B = A.copy()
    B.data = np.where(keep, B.data, 0.0)
    B.eliminate_zeros()
    B.sort_indices()
    return B, FilterInfo(eps_g, t, iters, b, A.nnz, B.nnz)


# --------------------------------------------------------------------------
# Algorithm 4.2
# --------------------------------------------------------------------------

@dataclasses.dataclass
class TaylorTerm:
    i: int
    nnz_raw: int
    nnz: int
    t: float
    iters: int
    products: int = 0


@dataclasses.dataclass
class SquareStep:
    i: int
    eps_g: float
    normF: float
    nnz_raw: int
    nnz: int
    t: float
    iters: int
    b: float
    products: int = 0


@dataclasses.dataclass
class OracleStats:
    n: int
    normH: float
    M: int
    N: int
    normal: bool
    a: float
    r0: float
    eps_g0: float
    taylor: List[TaylorTerm]
    steps: List[SquareStep]
    nnz_T0: int = 0
    nnz_out: int = 0


def product_count(A: sp.csr_matrix, B: sp.csr_matrix) -> int:
    """Number of scalar multiplications a_ik b_kj in the row-wise product A B (bookkeeping)."""
    return int(np.diff(B.indptr)[A.indices].sum()) if A.nnz else 0


def _canon(A) -> sp.csr_matrix:
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    return A


def taylor_phase(H0: sp.csr_matrix, M: int, eps_g0: float, e_r: float, max_iter: int = 100,
                 keep_terms: bool = False):
    """Algorithm 4.2 step 3 with the filtered recursion of Eq. (4.11).

    Returns (T^_0, list of TaylorTerm, list of the filtered terms S^_i if keep_terms).
    """
    S = _canon(H0)                     # S_1 = H_0 (not filtered)
    T0 = S.copy()
    terms: List[TaylorTerm] = []
    kept = [S.copy()] if keep_terms else None
    for i in range(2, M + 1):
        prev = S
        St = _canon(S @ H0)
        St.data = div_real(St.data, i)  # S~_i = S^_{i-1} H_0 / i
        S, info = filter_csr(St, eps_g0, e_r, max_iter)
        terms.append(TaylorTerm(i, St.nnz, S.nnz, info.t, info.iters, product_count(prev, H0)))
        if S.nnz == 0:
            break
        if keep_terms:
            kept.append(S.copy())
        T0 = _canon(T0 + S)            # T^_0^(i) = T^_0^(i-1) + S^_i
    return T0, terms, kept


def square_raw(T: sp.csr_matrix) -> sp.csr_matrix:
    """T~ = 2 T + T T (Eq. (2.7) / (4.15)), union pattern, unfiltered."""
    return _canon(_canon(T @ T) + 2.0 * T)


def norm_I_plus(T: sp.csr_matrix) -> float:
    """||I + T||_F, the estimate of ||F_i||_F used by the relative threshold."""
    return fro_norm(_canon(sp.identity(T.shape[0], format="csr") + T))


def squaring_phase(T0: sp.csr_matrix, N: int, a: float, r0: float, e_r: float, scale: str = "rel",
                   max_iter: int = 100, keep_iterates: bool = False):
    """Algorithm 4.2 step 4: N filtered incremental squarings."""
    T = T0
    steps: List[SquareStep] = []
    iterates = [T0.copy()] if keep_iterates else None
    for i in range(1, N + 1):
        ri = math.ldexp(r0, i)                 # r_i = 2 r_{i-1}
        Tprev = T
        Tt = square_raw(T)
        normF = norm_I_plus(Tt) if scale == "rel" else 1.0
        eps_g = a * ri * normF
        T, info = filter_csr(Tt, eps_g, e_r, max_iter)
        steps.append(SquareStep(i, eps_g, normF, Tt.nnz, T.nnz, info.t, info.iters, info.b, product_count(Tprev, Tprev)))
        if keep_iterates:
            iterates.append(T.copy())
    return T, steps, iterates


def plan_scalars(H: sp.csr_matrix, eps_tol: float, normal: Optional[bool] = None, n_extra: int = 50):
    """Algorithm 4.2 steps 1-3 scalars: ||H||, (M, N), a, r_0, eps_g^(0)."""
    normH = fro_norm(H)
    M, N = choose_MN(normH, eps_tol, n_extra)
    if normal is None:
        normal = is_normal(H)
    a = 1.0 / (1 + N) if normal else (1.0 / normH if normH > 0 else 1.0)
    x0 = math.ldexp(normH, -N)
    r0 = rho(M, x0) if M > 0 else 0.0
    eps_g0 = a * r0 / (M * math.exp(2.0 * x0)) if M > 0 else 0.0
    return normH, M, N, normal, a, r0, eps_g0


def expm(H, tau: float = 1.0, eps_tol: float = 1e-12, e_r: float = 0.1, square_scale: str = "rel",
         normal: Optional[bool] = None, max_iter: int = 100, n_extra: int = 50,
         keep: bool = False):
    """e^{tau H} by Algorithm 4.2.  Returns (E as scipy CSR, OracleStats[, trace])."""
    if not (eps_tol > 0.0 and math.isfinite(eps_tol)):
        raise OracleError("eps_tol must be positive and finite")
    H = _canon(H)
    n = H.shape[0]
    if tau != 1.0:
        H = H.copy()
        H.data = H.data * tau
    normH, M, N, normal, a, r0, eps_g0 = plan_scalars(H, eps_tol, normal, n_extra)
    stats = OracleStats(n, normH, M, N, normal, a, r0, eps_g0, [], [])
    eye = sp.identity(n, format="csr")
    if M == 0:
        E = _canon(eye)
        stats.nnz_out = E.nnz
        return (E, stats, None) if keep else (E, stats)
    H0 = H.copy()
    H0.data = scale_pow2(H0.data, -N)          # H_0 = H 2^-N (exact)
    T0, terms, kept_terms = taylor_phase(H0, M, eps_g0, e_r, max_iter, keep_terms=keep)
    stats.taylor = terms
    stats.nnz_T0 = T0.nnz
    T, steps, iterates = squaring_phase(T0, N, a, r0, e_r, square_scale, max_iter, keep_iterates=keep)
    stats.steps = steps
    E = _canon(eye + T)                        # e^H = I + T^_N
    stats.nnz_out = E.nnz
    if keep:
        return E, stats, {"H0": H0, "S": kept_terms, "T": iterates}
    return E, stats


# --------------------------------------------------------------------------
# Diagnostics used by the pins
# --------------------------------------------------------------------------

def bandwidth(A: sp.csr_matrix) -> int:
    """Natural-order bandwidth l(A) = l_1(A) + l_2(A), Eq. (3.1)."""
    A = sp.coo_matrix(A)
    nz = A.data != 0
    if not np.any(nz):
        return 0
    d = A.col[nz].astype(np.int64) - A.row[nz].astype(np.int64)
    return int(max(d.max(), 0) + max((-d).max(), 0))


# --------------------------------------------------------------------------
# Adjoint of the filtered method (masks frozen)
# --------------------------------------------------------------------------
#
# With the scaling N, the Taylor degree and every filter decision held fixed (they are
# piecewise constant in H), Algorithm 4.2 is a polynomial map H -> e^H:
#   S_1 = H_0,  S_i = P_i(S_{i-1} H_0 / i),  T_0 = sum_i S_i,
#   T_k = Q_k(2 T_{k-1} + T_{k-1}^2),  E = I + T_N,      H_0 = tau 2^-N H,
# where P_i, Q_k keep the stored pattern of the filtered S^_i, T^_k.  For L = <W, E> its
# reverse pass is, with Y = dL/dT_k on the pattern of T_k,
#   dL/dT_{k-1} = mask_{k-1}(2 Y + Y T_{k-1}^T + T_{k-1}^T Y)            (from Eq. (4.15)),
# then dL/dS_i = dL/dT_0 on the pattern of S_i, and for i = M'..2
#   dL/dS_{i-1} += mask(Y H_0^T) / i,   dL/dH_0 += mask_H(S_{i-1}^T Y) / i   (Y = dL/dS_i),
#   dL/dH_0 += dL/dS_1,  dL/dH = tau 2^-N dL/dH_0   (on the pattern of H).

def _ones(P: sp.csr_matrix) -> sp.csr_matrix:
    P = _canon(P)
    return sp.csr_matrix((np.ones(P.nnz), P.indices, P.indptr), shape=P.shape)


def restrict(X, P) -> sp.csr_matrix:
    """X on the stored pattern of P (entries of P's pattern missing from X are zeros)."""
    out = _canon(sp.csr_matrix(X).multiply(_ones(P)))
    return out


def square_adjoint(Y, Tp) -> sp.csr_matrix:
    """dL/dT_{k-1} = mask_{k-1}(2 Y + Y T_{k-1}^T + T_{k-1}^T Y) for T_k = Q_k(2 T_{k-1} + T_{k-1}^2)."""
    return restrict(2.0 * Y + Y @ Tp.T + Tp.T @ Y, Tp)


def adjoint(H, tau: float, eps_tol: float, W, e_r: float = 0.1, square_scale: str = "rel",
            normal: Optional[bool] = None, max_iter: int = 100):
    """dL/dH on the pattern of H for L = <W, e^{tau H}> (W sparse), masks frozen.

    Returns (G as scipy CSR with the pattern of H, E, stats, trace)."""
    H = _canon(H)
    E, st, tr = expm(H, tau, eps_tol, e_r, square_scale, normal, max_iter, keep=True)
    if st.M == 0:
        # ||tau H|| = 0: e^{tau H} = I + tau H + ..., so dL/dH = tau W on the pattern of H
        return restrict(sp.csr_matrix(W) * tau, H), E, st, tr
    H0, S, T = tr["H0"], tr["S"], tr["T"]
    G = restrict(W, T[-1])
    for k in range(len(T) - 1, 0, -1):
        G = square_adjoint(G, T[k - 1])
    GS = [restrict(G, Si) for Si in S]
    GH0 = restrict(sp.csr_matrix(H.shape), H)
    for i in range(len(S), 1, -1):
        Y = GS[i - 1]
        GS[i - 2] = _canon(GS[i - 2] + restrict(Y @ H0.T, S[i - 2]) / i)
        GH0 = _canon(GH0 + restrict(S[i - 2].T @ Y, H) / i)
    GH0 = _canon(GH0 + restrict(GS[0], H))
    GH = GH0 * (tau * math.ldexp(1.0, -st.N))
    return restrict(GH, H), E, st, tr


def forward_frozen(H, tau: float, N: int, S_masks, T_masks) -> sp.csr_matrix:
    """Algorithm 4.2 with N and every filter decision given: e^{tau H} as the polynomial map
    that the adjoint differentiates (S_masks[i-1] the pattern of S^_i, T_masks[k] of T^_k)."""
    H = _canon(H)
    H0 = H * (tau * math.ldexp(1.0, -N))
    S = restrict(H0, S_masks[0])
    T = S.copy()
    for i in range(2, len(S_masks) + 1):
        S = restrict(S @ H0 / i, S_masks[i - 1])
        T = _canon(T + S)
    T = restrict(T, T_masks[0])
    for k in range(1, len(T_masks)):
        T = restrict(2.0 * T + T @ T, T_masks[k])
    return _canon(sp.identity(H.shape[0], format="csr") + T)


# --------------------------------------------------------------------------
# Bandwidth bounds of the squaring iterates (Sec. 4.2, Eqs. 4.6-4.9)
# --------------------------------------------------------------------------

def power_norms(H, kmax: int) -> List[float]:
    """||H^k||_F for k = 1..kmax, from exact sparse powers (a library product per power)."""
    H = _canon(H)
    out = []
    P = H.copy()
    for k in range(1, kmax + 1):
        if k > 1:
            P = _canon(P @ H)
        out.append(fro_norm(P))
    return out


def h_refined(pnorms: List[float], M1: int, Np: int) -> float:
    """h_{M1,Np} = max over M1+1 <= k <= 2 M1 + 1 of ||(H 2^-Np)^k||^(1/k) (Sec. 4.2, from [11]),
    given pnorms[k-1] = ||H^k||."""
    best = 0.0
    for k in range(M1 + 1, 2 * M1 + 2):
        v = pnorms[k - 1]
        if v > 0.0:
            best = max(best, math.exp((math.log(v) - Np * k * math.log(2.0)) / k))
    return best


def alpha_hat(normH: float, M: int, N: int, i: int, pnorms: Optional[List[float]] = None,
              n1_max: int = 40, m1_max: int = 1000) -> int:
    """alpha^_i of Eq. (4.8) (pnorms None: ||H 2^{i-N} 2^{-N1}|| in rho) or of Eq. (4.9) (with
    pnorms[k-1] = ||H^k||: h_{M1, N+N1-i} in rho): the least M1 2^N1 with
    2^N1 rho(M1, .) <= r_i, where r_i = 2^i rho(M, ||H 2^-N||) (Eq. 4.6)."""
    ri = math.ldexp(rho(M, math.ldexp(normH, -N)), i)
    best = None
    for N1 in range(0, n1_max + 1):
        for M1 in range(1, m1_max + 1):
            if pnorms is None:
                x = math.ldexp(normH, i - N - N1)
            else:
                if 2 * M1 + 1 > len(pnorms):
                    break
                x = h_refined(pnorms, M1, N + N1 - i)
            if math.ldexp(rho(M1, x), N1) <= ri:
                c = M1 << N1
                if best is None or c < best:
                    best = c
                break
    if best is None:
        raise OracleError("no (M1, N1) meets r_i in the searched range")
    return best


def choose_MN_refined(normH: float, pnorms: List[float], eps_tol: float, n_extra: int = 50) -> Tuple[int, int]:
    """Eq. (4.20)'s rule with the refined norm of Sec. 4.2 in place of ||H 2^-N||: over N in
    [0, N0 + n_extra] (N0 = max(ceil(log2 ||H||), 0)), m(N) = the least M >= 1 (with 2M + 1 <= kmax)
    such that h_{M,N} <= 1 and 2^N rho(M, h_{M,N}) <= eps; minimise M 2^N, ties to the smaller M + N,
    then the smaller N."""
    if normH == 0.0:
        return 0, 0
    kmax = len(pnorms)
    N0 = max(ceil_log2(normH), 0)
    best = None
    for N in range(0, N0 + n_extra + 1):
        mN = None
        M = 1
        while 2 * M + 1 <= kmax:
            h = h_refined(pnorms, M, N)
            if h <= 1.0 and math.ldexp(rho(M, h), N) <= eps_tol:
                mN = M
                break
            M += 1
        if mN is None:
            continue
        key = (mN * 2 ** N, mN + N, N)
        if best is None or key < best[0]:
            best = (key, mN, N)
    if best is None:
        raise OracleError("no feasible (M, N) on the refined norm")
    return best[1], best[2]


def expm_refined(H, tau: float = 1.0, eps_tol: float = 1e-12, e_r: float = 0.1, kmax: int = 41):
    """Algorithm 4.2 with the refined scaling (reading of Sec. 4.2 / Eq. 4.9): (M, N) by
    choose_MN_refined on ||(tau H)^k||_F (exact sparse powers, k <= kmax), r_0 = rho(M, h_{M,N}) and
    eps_g^(0) = a r_0 / (M e^{2 h_{M,N}}); everything else as in expm()."""
    H = _canon(H)
    n = H.shape[0]
    if tau != 1.0:
        H = H.copy()
        H.data = H.data * tau
    normH = fro_norm(H)
    normal = is_normal(H)
    eye = sp.identity(n, format="csr")
    if normH == 0.0:
        return _canon(eye), (0, 0)
    pn = power_norms(H, kmax)
    M, N = choose_MN_refined(normH, pn, eps_tol)
    a = 1.0 / (1 + N) if normal else 1.0 / normH
    h = h_refined(pn, M, N)
    r0 = rho(M, h)
    eps_g0 = a * r0 / (M * math.exp(2.0 * h))
    H0 = H.copy()
    H0.data = scale_pow2(H0.data, -N)
    T0, terms, _ = taylor_phase(H0, M, eps_g0, e_r)
    T, steps, _ = squaring_phase(T0, N, a, r0, e_r)
    return _canon(eye + T), (M, N)
