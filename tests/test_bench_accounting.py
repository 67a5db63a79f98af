"""Host-side accounting of bench.py: the float64 flop count of the per-point solver by
route (the numerator of the solver's roofline), against the route costs it documents."""
import pytest

bench = pytest.importorskip("bench")


def test_solve_flops_by_route():
    n = 200
    full_inside = 5.0 / 3.0 * n ** 3
    full_outside = (1.0 / 3.0 + 2.0 / 3.0 + 1.0 / 3.0 + 2.0 + 4.0 / 3.0) * n ** 3
    assert bench.solve_flops([(n, n)], n) == pytest.approx(full_inside)
    assert bench.solve_flops([(n, n - 3)], n) == pytest.approx(full_outside)
    assert bench.solve_flops([(0, 0)], n) == 0.0
    # few dropped directions (3 d < r): reduction, back-transform + reflections, r x r pencil
    r, d = 190, 10
    assert bench.solve_flops([(r, r)], n) == pytest.approx(4.0 / 3.0 * n ** 3 + 4.0 / 3.0 * r ** 3 + 10.0 * n * n * d)
    # kept basis (3 d >= r): basis products instead
    r = 100
    assert bench.solve_flops([(r, r - 1)], n) == pytest.approx(
        4.0 / 3.0 * n ** 3 + 13.0 / 3.0 * r ** 3 + 4.0 * n * n * r + 2.0 * n * r * r)
    # additive over points
    pts = [(n, n), (0, 0), (190, 190), (100, 99)]
    assert bench.solve_flops(pts, n) == pytest.approx(sum(bench.solve_flops([p], n) for p in pts))
