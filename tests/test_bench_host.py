"""Host-side accounting of the benchmark (CPU only): the algorithmic flop
count per cell and vector that the roofline divides by.

The trilinear-cell count is the one the hot-path scope fixes per workload
(4^3 p=4 n_q=6: 29,928; p=6 n_q=8: 95,200; p=8 n_q=10: 233,560).  Box cells
have a diagonal metric, so their quadrature-point operation is three
scalings plus the value scaling, 4 flops per point instead of 16, which the
count must differ by exactly 12 n_q^3.  Checked against a pass-by-pass tally
of the sum-factorisation sweeps written out independently below."""
import bench


def _tally(np_, nq, box):
    """2 flops per multiply-add, sweep by sweep: forward N along x, y, z; the
    three D~ gradients on the n_q^3 grid; their transposes; backward N^T."""
    f = 0
    f += 2 * (np_ * np_) * nq * np_      # N along x: n_p^2 lines, n_q outputs of n_p terms
    f += 2 * (nq * np_) * nq * np_       # N along y
    f += 2 * (nq * nq) * nq * np_        # N along z
    f += 3 * 2 * (nq * nq) * nq * nq     # D~ along x, y, z
    f += 3 * 2 * (nq * nq) * nq * nq     # D~^T along x, y, z
    f += 2 * (nq * nq) * np_ * nq        # N^T along z
    f += 2 * (nq * np_) * np_ * nq       # N^T along y
    f += 2 * (np_ * np_) * np_ * nq      # N^T along x
    f += (4 if box else 16) * nq ** 3    # point operation
    return f


def test_flops_per_cell_vec_matches_scope_table():
    assert bench.flops_per_cell_vec(5, 6, box=False) == 29928
    assert bench.flops_per_cell_vec(7, 8, box=False) == 95200
    assert bench.flops_per_cell_vec(9, 10, box=False) == 233560


def test_box_cells_count_the_diagonal_metric():
    for np_, nq in ((2, 3), (5, 6), (7, 8), (7, 9), (9, 10)):
        full = bench.flops_per_cell_vec(np_, nq, box=False)
        box = bench.flops_per_cell_vec(np_, nq, box=True)
        assert full - box == 12 * nq ** 3
        assert box == _tally(np_, nq, True) and full == _tally(np_, nq, False)
    assert bench.flops_per_cell_vec(7, 8) == 89056
