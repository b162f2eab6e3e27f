"""The seeded input generators shared by the oracle side and the GPU side:
storage types, ranges, determinism and the structure each workload promises
(triangular systems with a non-zero diagonal, the batched size grid)."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("e", range(2, 11))
def test_elements_range_type_and_coverage(e):
    x = workloads.elements(np.random.default_rng(e), e, (64, 300))
    assert x.dtype == (np.uint8 if e <= 8 else np.uint16)
    assert int(x.min()) >= 0 and int(x.max()) < (1 << e)
    if e <= 8:  # 19200 draws cover every one of at most 256 values
        assert len(np.unique(x)) == 1 << e


def test_field_polynomials_have_degree_e():
    for e, f in workloads.FIELD_POLY.items():
        assert f >> e == 1 and f & 1  # x^e term, no higher term, non-zero constant


def test_random_problem_is_seeded():
    A1, B1, C1 = workloads.random_problem(4, 10, 7, 5, seed=3, with_c=True)
    A2, B2, C2 = workloads.random_problem(4, 10, 7, 5, seed=3, with_c=True)
    A3, B3, C3 = workloads.random_problem(4, 10, 7, 5, seed=3)
    assert A1.shape == (10, 5) and B1.shape == (5, 7) and C1.shape == (10, 7) and C3 is None
    assert np.array_equal(A1, A2) and np.array_equal(B1, B2) and np.array_equal(C1, C2)
    assert np.array_equal(A1, A3) and np.array_equal(B1, B3)  # drawing C does not change A, B
    A4, _, _ = workloads.random_problem(4, 10, 7, 5, seed=4)
    assert not np.array_equal(A1, A4)


def test_workload_row_panel_matches_the_full_inputs():
    w = workloads.WORKLOADS[1]
    A, B, C = w.inputs()
    Ap, Bp, Cp = w.inputs(rows=slice(100, 140))
    assert C is None and Cp is None
    assert np.array_equal(Ap, A[100:140]) and np.array_equal(Bp, B)
    assert w.field_ops == 2.0 * 512 ** 3 and w.f == 0x7


@pytest.mark.parametrize("upper", [True, False])
def test_triangular_system_structure(upper):
    T, B = workloads.triangular_system(4, 50, 7, seed=5, upper=upper)
    assert T.shape == (50, 50) and B.shape == (50, 7)
    off = np.tril(T, -1) if upper else np.triu(T, 1)
    assert not off.any()
    assert (np.diag(T) != 0).all() and int(T.max()) < 16


def test_batched_instances_follow_the_grid():
    seen_e = set()
    for j in range(200):
        e, f, m, n, k, A, B = workloads.batched_instance(j)
        assert 2 <= e <= 8 and f == workloads.FIELD_POLY[e]
        for d in (m, n, k):
            assert d % 32 == 0 and 32 <= d <= 1024
        assert A.shape == (m, k) and B.shape == (k, n) and int(A.max()) < (1 << e)
        assert workloads.batched_instance(j, dims_only=True)[:5] == (e, f, m, n, k)
        seen_e.add(e)
    assert seen_e == set(range(2, 9))


def test_echelon_matrices_are_seeded_and_in_range():
    for name, (e, m, n, seed) in workloads.ECHELON_WORKLOADS.items():
        if m * n > 2 ** 22:
            continue
        X = workloads.echelon_matrix(e, m, n, seed)
        assert X.shape == (m, n) and int(X.max()) < (1 << e)
        assert np.array_equal(X, workloads.echelon_matrix(e, m, n, seed))
