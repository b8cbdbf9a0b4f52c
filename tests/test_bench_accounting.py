"""The algorithmic byte counts behind the bench line's roofline, checked against
an explicit list of the buffers each pass must read and write once (CPU only)."""
import bench

N = 128
V = N ** 3
C = 6
NXH = N // 2 + 1


def spectrum_bytes(b):
    """One half spectrum of all components: c * nz * ny * (nx/2+1) complex values."""
    return C * N * N * NXH * 2 * b


def field_bytes(b):
    return C * V * b


def test_x_forward_reads_three_fields_writes_two_and_the_spectrum():
    for b in (4, 8):
        expected = 3 * field_bytes(b) + 2 * field_bytes(b) + spectrum_bytes(b)
        assert abs(bench.pass_traffic("x_forward", V, C, N, NXH, 21, b) - expected) < 1e-6 * expected


def test_y_passes_read_and_write_the_spectrum_once():
    for kind in ("y_forward", "y_inverse"):
        assert bench.pass_traffic(kind, V, C, N, NXH, 21, 4) == 2 * spectrum_bytes(4)


def test_z_pass_adds_the_symmetric_table_once():
    table = N * N * NXH * 21 * 4  # c(c+1)/2 = 21 coefficients per frequency
    assert bench.pass_traffic("z_gamma", V, C, N, NXH, 21, 4) == 2 * spectrum_bytes(4) + table
    assert bench.pass_traffic("z_gamma", V, C, N, NXH, 0, 4) == 2 * spectrum_bytes(4)  # computed in the kernel


def test_x_inverse_reads_spectrum_and_p_writes_q_and_reads_the_phase_byte():
    expected = spectrum_bytes(4) + 2 * field_bytes(4) + C * V  # one phase byte per voxel-component
    assert bench.pass_traffic("x_inverse_local", V, C, N, NXH, 21, 4) == expected


def test_cg_update_reads_r_q_writes_r():
    assert bench.pass_traffic("cg_update", V, C, N, NXH, 21, 4) == 3 * field_bytes(4)


def test_one_fp32_iteration_moves_about_81_bytes_per_voxel_component():
    kinds = ("x_forward", "y_forward", "z_gamma", "y_inverse", "x_inverse_local", "cg_update")
    total = sum(bench.pass_traffic(k, V, C, N, NXH, 21, 4) for k in kinds)
    assert 80.0 < total / (C * V) < 82.0
