"""CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The product library never loads it and shares no code,
header, table or constant generator with it.

Two layers:
  * `sic_oracle.c` (plain C, FP64, compiled with -ffp-contract=off): kernel entries,
    reverse-maximin ordering, later-ordered nearest neighbours, grouping, the
    single- and multiple-target greedy selections in the paper's Cholesky form,
    the KL-optimal fill by dense solves, and a CSC product;
  * numpy code in this file: the naive re-factorising greedy forms, exhaustive
    subset search, dense log-determinants, the picks' FP64 conditional variances,
    the reverse-Cholesky aggregated fill and the KL assembly.  numpy's Cholesky / slogdet serve as library primitives.

Parity pins for each function live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from itertools import combinations

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sic_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction) into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Kernel(C.Structure):
    """Matern kernel parameters; nu_x2 = 2*nu in {1, 3, 5}."""
    _fields_ = [("dim", C.c_int32), ("nu_x2", C.c_int32), ("length_scale", C.c_double),
                ("variance", C.c_double), ("nugget", C.c_double),
                ("dense", C.POINTER(C.c_double)), ("dense_ld", C.c_int64)]


def kernel(dim, nu_x2, length_scale, variance=1.0, nugget=0.0) -> Kernel:
    return Kernel(int(dim), int(nu_x2), float(length_scale), float(variance), float(nugget), None, 0)


def dense_kernel(theta: np.ndarray):
    """A 'kernel' whose entries are read from an explicit SPD matrix (rows = positions).
    Returns (kernel, dummy points); keep the returned matrix alive while in use."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    n = theta.shape[0]
    kp = Kernel(1, 1, 1.0, float(np.max(np.diag(theta))), 0.0, theta.ctypes.data_as(C.POINTER(C.c_double)), n)
    kp._keep = theta
    return kp, np.zeros((n, 1))


def exhaustion_floor(kp: Kernel) -> float:
    """A candidate is exhausted once its conditional variance falls below this value:
    half the nugget (every true conditional variance is at least the nugget), or
    1e-14 * variance when there is no nugget."""
    return 0.5 * kp.nugget if kp.nugget > 0 else 1e-14 * kp.variance


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        d, i32, i64 = C.c_double, C.c_int32, C.c_int64
        pd, pi32, pi64 = P(d), P(i32), P(i64)
        pk = P(Kernel)
        L.or_matern.argtypes = [pk, d]; L.or_matern.restype = d
        L.or_theta.argtypes = [pk, pd, i64, i64]; L.or_theta.restype = d
        L.or_maximin.argtypes = [pd, i64, C.c_int, pi64, pd]; L.or_maximin.restype = None
        L.or_knn_later.argtypes = [pd, i64, C.c_int, pi64, i32, i64, i32, pi32]; L.or_knn_later.restype = i32
        L.or_group.argtypes = [pd, pd, i64, C.c_int, i32, d, i32, i32, pi64, pi64]; L.or_group.restype = i64
        L.or_select_single.argtypes = [pk, pd, i64, pi32, i32, i32, d, pi32, pi32, pd, pd, pd]
        L.or_select_single.restype = i32
        L.or_select_multi.argtypes = [pk, pd, i64, i32, pi32, i32, i32, d, pi32, pi32, pd, pd]
        L.or_select_multi.restype = i32
        L.or_fill_set.argtypes = [pk, pd, pi64, i32, pd]; L.or_fill_set.restype = d
        L.or_fill_column.argtypes = [pk, pd, i64, pi32, i32, pi64, pd]; L.or_fill_column.restype = d
        L.or_fill_member.argtypes = [pk, pd, i64, i32, i32, pi32, i32, pi64, pd]; L.or_fill_member.restype = d
        L.or_theta_matrix.argtypes = [pk, pd, pi64, i32, pd]; L.or_theta_matrix.restype = None
        L.or_apply_factor.argtypes = [i64, pi64, pi32, pd, i32, pd, pd, i32]; L.or_apply_factor.restype = None
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# ------------------------------------------------------------------- kernel --

def matern(kp: Kernel, r: float) -> float:
    return lib().or_matern(C.byref(kp), float(r))


def theta_matrix(kp: Kernel, pts, idx) -> np.ndarray:
    """Dense Theta restricted to rows/columns idx (positions into pts)."""
    pts = _f64(pts)
    idx = _i64(idx)
    out = np.empty((len(idx), len(idx)))
    lib().or_theta_matrix(C.byref(kp), _p(pts, C.c_double), _p(idx, C.c_int64), len(idx), _p(out, C.c_double))
    return out


# --------------------------------------------------------------------- prep --

def maximin(pts):
    """Reverse-maximin ordering (eq. maximin).  Returns (order, ell2): order[pos] = point index."""
    pts = _f64(pts)
    n, dim = pts.shape
    order = np.empty(n, np.int64)
    ell2 = np.empty(n)
    lib().or_maximin(_p(pts, C.c_double), n, dim, _p(order, C.c_int64), _p(ell2, C.c_double))
    return order, ell2


def knn_later(pts, targets, first: int, n_cand: int) -> np.ndarray:
    """The n_cand positions >= first nearest (min over targets) to the targets."""
    pts = _f64(pts)
    t = _i64(np.atleast_1d(targets))
    out = np.empty(max(n_cand, 1), np.int32)
    cnt = lib().or_knn_later(_p(pts, C.c_double), pts.shape[0], pts.shape[1], _p(t, C.c_int64), len(t),
                             int(first), int(n_cand), _p(out, C.c_int32))
    return out[:cnt].copy()


def column_candidates(pts, n_cand: int, threads: int | None = None):
    """CSR candidate lists of every column i: its n_cand nearest later positions."""
    n = pts.shape[0]
    pts = _f64(pts)

    def one(i):
        return knn_later(pts, [i], i + 1, n_cand)

    with ThreadPoolExecutor(threads or os.cpu_count()) as ex:
        lists = list(ex.map(one, range(n), chunksize=256))
    ptr = np.zeros(n + 1, np.int64)
    ptr[1:] = np.cumsum([len(x) for x in lists])
    idx = np.concatenate(lists).astype(np.int32) if n else np.zeros(0, np.int32)
    return ptr, idx


def group(pts, ell2, K: int, lambda_: float = 1.5, mmin: int = 8, mmax: int = 64):
    """Supernodes by the Section 6.1 rule plus the small-group merge.  Returns (members,
    grp_ptr): members lists the old positions in the renumbered order; group g is
    members[grp_ptr[g]:grp_ptr[g+1]]."""
    pts = _f64(pts)
    ell2 = _f64(ell2)
    n = pts.shape[0]
    members = np.empty(n, np.int64)
    gp = np.empty(n + 1, np.int64)
    ng = lib().or_group(_p(pts, C.c_double), _p(ell2, C.c_double), n, pts.shape[1], int(K),
                        float(lambda_) ** 2, int(mmin), int(mmax), _p(members, C.c_int64), _p(gp, C.c_int64))
    return members, gp[:ng + 1].copy()


def group_candidates(pts, grp_ptr, n_cand: int, threads: int | None = None):
    """CSR candidate lists of each group (positions after the group, nearest to any member)."""
    pts = _f64(pts)
    ng = len(grp_ptr) - 1

    def one(g):
        a, b = int(grp_ptr[g]), int(grp_ptr[g + 1])
        return knn_later(pts, np.arange(a, b), b, n_cand)

    with ThreadPoolExecutor(threads or os.cpu_count()) as ex:
        lists = list(ex.map(one, range(ng), chunksize=64))
    ptr = np.zeros(ng + 1, np.int64)
    ptr[1:] = np.cumsum([len(x) for x in lists])
    idx = np.concatenate(lists).astype(np.int32) if ng else np.zeros(0, np.int32)
    return ptr, idx


# ---------------------------------------------------------------- selection --

def select_single(kp: Kernel, pts, target: int, cand, k: int, floor=None, forced=None):
    """Single-target greedy selection (Cholesky approach).  forced[t] >= 0 replays a pick
    given as an index into cand.  Returns dict(sel, best, chosen, vtar)."""
    pts = _f64(pts)
    cand = _i32(cand)
    Cn = len(cand)
    floor = exhaustion_floor(kp) if floor is None else floor
    sel = np.full(max(k, 1), -1, np.int32)
    best = np.zeros(max(k, 1))
    chosen = np.zeros(max(k, 1))
    vtar = np.zeros(k + 1)
    fp = None
    if forced is not None:
        f = np.full(max(k, 1), -1, np.int32)
        f[:len(forced)] = forced
        fp = _p(f, C.c_int32)
    cnt = lib().or_select_single(C.byref(kp), _p(pts, C.c_double), int(target), _p(cand, C.c_int32), Cn, int(k),
                                 float(floor), fp, _p(sel, C.c_int32), _p(best, C.c_double),
                                 _p(chosen, C.c_double), _p(vtar, C.c_double))
    return dict(sel=sel[:cnt].copy(), best=best[:cnt].copy(), chosen=chosen[:cnt].copy(), vtar=vtar[:cnt + 1].copy())


def select_multi(kp: Kernel, pts, g0: int, m: int, cand, k: int, floor=None, forced=None):
    """Multiple-target greedy selection with two partial Cholesky factors.  Targets are
    positions g0 .. g0+m-1.  Returns dict(sel, best, chosen); raises on a non-PD target block."""
    pts = _f64(pts)
    cand = _i32(cand)
    floor = exhaustion_floor(kp) if floor is None else floor
    sel = np.full(max(k, 1), -1, np.int32)
    best = np.zeros(max(k, 1))
    chosen = np.zeros(max(k, 1))
    fp = None
    if forced is not None:
        f = np.full(max(k, 1), -1, np.int32)
        f[:len(forced)] = forced
        fp = _p(f, C.c_int32)
    cnt = lib().or_select_multi(C.byref(kp), _p(pts, C.c_double), int(g0), int(m), _p(cand, C.c_int32), len(cand),
                                int(k), float(floor), fp, _p(sel, C.c_int32), _p(best, C.c_double),
                                _p(chosen, C.c_double))
    if cnt < 0:
        raise np.linalg.LinAlgError("target block not positive definite")
    return dict(sel=sel[:cnt].copy(), best=best[:cnt].copy(), chosen=chosen[:cnt].copy())


def select_single_naive(kp: Kernel, pts, target: int, cand, k: int, floor=None):
    """Naive greedy (O(C k^4)): at every step re-factorise Theta_{S+j,S+j} for each
    unselected j and take the j of least target conditional variance (eq. cond_cov).
    A candidate is skipped when its own conditional variance given S is below floor."""
    floor = exhaustion_floor(kp) if floor is None else floor
    cand = list(int(c) for c in cand)
    S: list[int] = []
    out_v = []
    for _ in range(k):
        best_j, best_v = None, None
        for j in cand:
            if j in S:
                continue
            idx = S + [j]
            K = theta_matrix(kp, pts, idx)
            b = theta_matrix(kp, pts, [target] + idx)[0, 1:]
            # conditional variance of j given S (exhaustion rule)
            if S:
                Ks = K[:-1, :-1]
                kj = K[:-1, -1]
                vj = K[-1, -1] - kj @ np.linalg.solve(Ks, kj)
            else:
                vj = K[-1, -1]
            if vj < floor:
                continue
            G = np.linalg.cholesky(K)
            w = np.linalg.solve(G, b)
            v = theta_matrix(kp, pts, [target])[0, 0] - w @ w
            if best_v is None or v < best_v:
                best_j, best_v = j, v
        if best_j is None:
            break
        S.append(best_j)
        out_v.append(best_v)
    return np.array(S, np.int32), np.array(out_v)


def logdet_cond(kp: Kernel, pts, P, S) -> float:
    """logdet Theta_{P,P | S} by dense Cholesky of the joint matrix."""
    P = list(P)
    S = list(S)
    K = theta_matrix(kp, pts, S + P)
    s = len(S)
    A = K[s:, s:]
    if s:
        B = K[:s, s:]
        A = A - B.T @ np.linalg.solve(K[:s, :s], B)
    return float(np.linalg.slogdet(A)[1])


def select_multi_naive(kp: Kernel, pts, g0: int, m: int, cand, k: int, floor=None):
    """Naive multiple-target greedy: each step re-factorises and takes
    argmin_j logdet Theta_{P,P | S + j} (Section 5.2 objective, D-optimal design)."""
    floor = exhaustion_floor(kp) if floor is None else floor
    P = list(range(g0, g0 + m))
    S: list[int] = []
    vals = []
    for _ in range(k):
        best_j, best_v = None, None
        for j in cand:
            j = int(j)
            if j in S:
                continue
            # exhaustion: conditional variance of j given P and S
            K = theta_matrix(kp, pts, P + S + [j])
            n0 = len(P) + len(S)
            vj = K[-1, -1] - K[:n0, -1] @ np.linalg.solve(K[:n0, :n0], K[:n0, -1])
            if vj < floor:
                continue
            v = logdet_cond(kp, pts, P, S + [j])
            if best_v is None or v < best_v:
                best_j, best_v = j, v
        if best_j is None:
            break
        S.append(best_j)
        vals.append(best_v)
    return np.array(S, np.int32), np.array(vals)


def pivot_variances(kp: Kernel, pts, P, picks):
    """FP64 side state of a selection: for the t-th pick q_t of a unit with targets P,
    (var1[t], var2[t]) = (Theta_{q_t q_t | q_0..q_t-1}, Theta_{q_t q_t | q_0..q_t-1, P}),
    the pivot's conditional variance without and with the targets, each by one dense
    Schur complement (the plain definition of a conditional variance).  The pick's
    decrease of logdet Theta_{PP|I} is log(var1 / var2) (eq. greedy_mult)."""
    P = [int(x) for x in P]
    picks = [int(x) for x in picks]
    var1 = np.zeros(len(picks))
    var2 = np.zeros(len(picks))
    for t, q in enumerate(picks):
        for out, cond in ((var1, picks[:t]), (var2, P + picks[:t])):
            K = theta_matrix(kp, pts, cond + [q])
            c = len(cond)
            out[t] = K[c, c] - (K[:c, c] @ np.linalg.solve(K[:c, :c], K[:c, c]) if c else 0.0)
    return var1, var2


def brute_force_subset(kp: Kernel, pts, target: int, cand, k: int):
    """Exhaustive search over all k-subsets of cand for the least target conditional variance."""
    best_S, best_v = None, None
    tt = theta_matrix(kp, pts, [target])[0, 0]
    for S in combinations([int(c) for c in cand], k):
        K = theta_matrix(kp, pts, list(S))
        b = theta_matrix(kp, pts, [target] + list(S))[0, 1:]
        v = tt - b @ np.linalg.solve(K, b)
        if best_v is None or v < best_v:
            best_S, best_v = S, v
    return best_S, best_v


# --------------------------------------------------------------------- fill --

def fill_column(kp: Kernel, pts, i: int, sel):
    """eq. L_col for column i with selections sel: (rows, values, log v_i); rows start with i
    then ascend."""
    pts = _f64(pts)
    sel = _i32(sel)
    rows = np.empty(len(sel) + 1, np.int64)
    L = np.empty(len(sel) + 1)
    lv = lib().or_fill_column(C.byref(kp), _p(pts, C.c_double), int(i), _p(sel, C.c_int32), len(sel),
                              _p(rows, C.c_int64), _p(L, C.c_double))
    return rows, L, lv


def fill_member(kp: Kernel, pts, g0: int, m: int, a: int, sel):
    """Aggregated fill of member a of the group g0..g0+m-1 (dense solve per member)."""
    pts = _f64(pts)
    sel = _i32(sel)
    n = (m - a) + len(sel)
    rows = np.empty(n, np.int64)
    L = np.empty(n)
    lv = lib().or_fill_member(C.byref(kp), _p(pts, C.c_double), int(g0), int(m), int(a), _p(sel, C.c_int32),
                              len(sel), _p(rows, C.c_int64), _p(L, C.c_double))
    return rows, L, lv


def fill_group_reverse_chol(kp: Kernel, pts, g0: int, m: int, sel):
    """Second, independent aggregated fill (Appendix A.4, eq. L_precision): U = P chol(P Theta P) P
    with P the order-reversing permutation, so U U^T = Theta_{s,s} with U upper triangular;
    L = U^{-T} is lower triangular with L L^T = Theta_{s,s}^{-1}.  Returns (rows, Lmat[:, :m], logv)."""
    rows = list(range(g0, g0 + m)) + sorted(int(s) for s in sel)
    T = theta_matrix(kp, pts, rows)
    Pr = T[::-1, ::-1]
    Gr = np.linalg.cholesky(Pr)
    U = Gr[::-1, ::-1]
    Lm = np.linalg.inv(U).T
    logv = -2.0 * np.log(np.diag(Lm)[:m])
    return np.array(rows, np.int64), Lm[:, :m], logv


def logdet_theta(kp: Kernel, pts) -> float:
    """logdet of the full kernel matrix by dense Cholesky (library primitive)."""
    n = pts.shape[0]
    K = theta_matrix(kp, pts, np.arange(n))
    G = np.linalg.cholesky(K)
    return float(2.0 * np.sum(np.log(np.diag(G))))


def kl_from_logv(sum_logv: float, logdet: float) -> float:
    """KL(N(0,Theta) || N(0,(L L^T)^{-1})) = (sum_i log v_i - logdet Theta) / 2 (eq. obj_chol)."""
    return 0.5 * (sum_logv - logdet)


# ------------------------------------------------------------ whole factors --

def factor_columns(kp: Kernel, pts, sel_lists, threads: int | None = None):
    """CSC factor from per-column selections (column i's set = i + sel_lists[i])."""
    n = pts.shape[0]
    pts = _f64(pts)

    def one(i):
        return fill_column(kp, pts, i, sel_lists[i])

    with ThreadPoolExecutor(threads or os.cpu_count()) as ex:
        res = list(ex.map(one, range(n), chunksize=64))
    col_ptr = np.zeros(n + 1, np.int64)
    col_ptr[1:] = np.cumsum([len(r[0]) for r in res])
    row_idx = np.concatenate([r[0] for r in res]).astype(np.int32)
    val = np.concatenate([r[1] for r in res])
    logv = np.array([r[2] for r in res])
    return col_ptr, row_idx, val, logv


def factor_groups(kp: Kernel, pts, grp_ptr, sel_lists, threads: int | None = None):
    """CSC factor from per-group selections (member columns by the dense per-member solve)."""
    pts = _f64(pts)
    n = pts.shape[0]
    jobs = []
    for g in range(len(grp_ptr) - 1):
        g0, g1 = int(grp_ptr[g]), int(grp_ptr[g + 1])
        for a in range(g1 - g0):
            jobs.append((g0, g1 - g0, a, sel_lists[g]))

    def one(j):
        return fill_member(kp, pts, *j)

    with ThreadPoolExecutor(threads or os.cpu_count()) as ex:
        res = list(ex.map(one, jobs, chunksize=64))
    assert len(res) == n
    col_ptr = np.zeros(n + 1, np.int64)
    col_ptr[1:] = np.cumsum([len(r[0]) for r in res])
    row_idx = np.concatenate([r[0] for r in res]).astype(np.int32)
    val = np.concatenate([r[1] for r in res])
    logv = np.array([r[2] for r in res])
    return col_ptr, row_idx, val, logv


def apply_factor(n, col_ptr, row_idx, val, op: int, x):
    """y = L x (op 0), L^T x (op 1) or L L^T x (op 2); x is n x nrhs."""
    x = _f64(x)
    if x.ndim == 1:
        x = x[:, None]
    nrhs = x.shape[1]
    y = np.empty_like(x)
    col_ptr = _i64(col_ptr)
    row_idx = _i32(row_idx)
    val = _f64(val)
    lib().or_apply_factor(int(n), _p(col_ptr, C.c_int64), _p(row_idx, C.c_int32), _p(val, C.c_double), int(op),
                          _p(x, C.c_double), _p(y, C.c_double), nrhs)
    return y
