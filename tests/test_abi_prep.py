"""CPU tests of the C-ABI library: it loads, exports every symbol include/sic.h declares,
rejects bad arguments on the host, and its host input preparation reproduces the
oracle's brute-force ordering, candidate lists and groups exactly."""
import os
import re

import numpy as np
import pytest

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sic():
    from paper_2307_11648_gb300 import build, sic as s
    build.build()
    return s


def test_exports_every_declared_symbol(sic):
    hdr = open(os.path.join(ROOT, "include", "sic.h")).read()
    declared = sorted(set(re.findall(r"\b(sic_[a-z0-9_]+)\s*\(", hdr)))
    assert declared, "no declarations parsed"
    L = sic.lib()
    missing = [d for d in declared if not hasattr(L, d)]
    assert not missing, missing
    assert sorted(sic.EXPORTS) == declared


def test_status_strings_and_floor(sic):
    assert sic.status_string(sic.SIC_OK) == "ok"
    assert "positive definite" in sic.status_string(sic.SIC_ERR_NOT_PD)
    assert sic.exhaustion_floor(sic.kernel(2, 3, 0.1, 1.0, 1e-6)) == 0.5e-6
    assert sic.exhaustion_floor(sic.kernel(2, 3, 0.1, 2.0, 0.0)) == 2e-14


def test_workspace_queries(sic):
    assert sic.select_single_workspace(1000, 10, sic.SIC_FP64) == 8 * (10 * 1000 + 2000)
    assert sic.factor_nnz_workspace(5000) >= 8 * (5001 // 1024 + 1)
    assert sic.apply_factor_workspace(100, 4, sic.SIC_OP_LLT) == 100 * 4 * 8
    assert sic.apply_factor_workspace(100, 4, sic.SIC_OP_L) == 0


def test_host_argument_errors(sic):
    with pytest.raises(sic.SicError) as e:
        sic.prep_maximin(np.zeros((5, 4)))
    assert e.value.code == sic.SIC_ERR_INVALID
    bad = synthetic.points(10, 2, 0)
    bad[3, 1] = np.nan
    with pytest.raises(sic.SicError):
        sic.prep_maximin(bad)


@pytest.mark.parametrize("n,dim,seed", [(1, 2, 0), (2, 2, 0), (700, 1, 3), (2500, 2, 1), (1800, 3, 2)])
def test_prep_matches_oracle(sic, oracle_lib, n, dim, seed):
    oracle = oracle_lib
    pts = synthetic.points(n, dim, seed)
    o1, e1 = sic.prep_maximin(pts)
    o2, e2 = oracle.maximin(pts)
    assert np.array_equal(o1, o2)
    assert np.array_equal(e1, e2)
    P = pts[o1]
    for C in [1, 17, 64]:
        p1, i1 = sic.prep_candidates_columns(P, C)
        p2, i2 = oracle.column_candidates(P, C)
        assert np.array_equal(p1, p2) and np.array_equal(i1, i2)
    m1, g1 = sic.prep_groups(P, e1, 32, 1.5, 4, 32)
    m2, g2 = oracle.group(P, e2, 32, 1.5, 4, 32)
    assert np.array_equal(m1, m2) and np.array_equal(g1, g2)
    P2 = P[m1]
    c1, j1 = sic.prep_candidates_groups(P2, g1, 50)
    c2, j2 = oracle.group_candidates(P2, g1, 50)
    assert np.array_equal(c1, c2) and np.array_equal(j1, j2)


def test_prep_grid_points_and_ties(sic, oracle_lib):
    """Points on an exact grid have many equal distances: the tie rules (lowest point
    index in the ordering, lowest position among candidates) must agree exactly."""
    oracle = oracle_lib
    g = np.arange(24) / 24.0
    pts = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2).copy()
    o1, e1 = sic.prep_maximin(pts)
    o2, e2 = oracle.maximin(pts)
    assert np.array_equal(o1, o2) and np.array_equal(e1, e2)
    P = pts[o1]
    p1, i1 = sic.prep_candidates_columns(P, 30)
    p2, i2 = oracle.column_candidates(P, 30)
    assert np.array_equal(i1, i2)


def test_package_modules_import():
    """Every module of the package and bench.py parse and import on a host without a GPU
    (the library itself is only loaded on first use)."""
    import ast
    import importlib
    import os
    for mod in ["sic", "pipeline", "learned", "gp", "build"]:
        importlib.import_module(f"paper_2307_11648_gb300.{mod}")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for f in ["bench.py", "__graft_entry__.py"]:
        ast.parse(open(os.path.join(root, f)).read())


@pytest.mark.parametrize("seed", [0, 1])
def test_prep_candidates_partial_brute_force(sic, oracle_lib, seed):
    """Candidates of nonadjacent groups: the n_cand points after the first member, members
    excluded, by (least squared distance to a member, position) -- checked by brute force on
    the groups of the Section 6.1 rule kept in the original ordering."""
    oracle = oracle_lib
    pts = synthetic.points(1500, 2, 40 + seed)
    order, ell2 = sic.prep_maximin(pts)
    P = np.ascontiguousarray(pts[order])
    members, gp = sic.prep_groups(P, ell2, 32, 1.5, 4, 32)
    ptr, idx = sic.prep_candidates_partial(P, members, gp, 40)
    nonadjacent = 0
    for g in range(len(gp) - 1):
        mem = members[gp[g]:gp[g + 1]]
        nonadjacent += int(mem[-1] - mem[0] + 1 != len(mem))
        d = ((P[:, None, :] - P[None, mem, :]) ** 2).sum(-1).min(1)
        ok = [j for j in range(len(P)) if j > mem[0] and j not in set(mem.tolist())]
        want = sorted(ok, key=lambda j: (d[j], j))[:40]
        assert idx[ptr[g]:ptr[g + 1]].tolist() == want, g
    assert nonadjacent > 0
