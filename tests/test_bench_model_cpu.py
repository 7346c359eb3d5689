"""Host logic of bench.py's flow byte model: the u* update is named for the
kernel that runs it and moves the same bytes on both viscous-solve paths;
the Fourier path's scaling pass is counted per Fourier substep."""
import bench


def test_flow_bytes_by_solve_path():
    n = (64, 48, 40)
    N = n[0] * n[1] * n[2]
    NC = n[2] * n[1] * (n[0] // 2 + 1)
    real = bench.flow_bytes(n, (4, 3, 3))
    fourier = bench.flow_bytes(n, (-1, -1, -1))
    mixed = bench.flow_bytes(n, (-1, 7, -1))
    assert "cn_solve" in real and "cn_scale" not in real and "add" not in real
    assert "add" in fourier and fourier["cn_scale"] == 3 * 3 * NC * 16
    assert "update" in mixed and mixed["cn_scale"] == 2 * 3 * NC * 16
    assert real["cn_solve"] == fourier["add"] == mixed["update"] == 3 * 36 * N
    for d in (real, fourier, mixed):
        assert d["rhs"] == (40 + 2 * 52) * N       # substep 0 reads no H_prev
        assert d["div"] == 3 * 28 * N and d["project"] == 3 * 48 * N
        assert d["poisson_scale"] == 3 * NC * 16
