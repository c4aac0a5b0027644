"""bench.py's algorithmic byte counts (the numerators of the reported roofline fractions) are
consistent between the fused and the two-pass interpolation, and scale with the value size."""
import bench


def _sizes(split: bool):
    dev = {k: {"col_bits": 16, "entries": n} for k, n in
           (("adjacency", 14_779_600), ("precorrection", 215_306_854), ("projection", 63_667_200))}
    return {"Np": 994_800, "dims": [128, 128, 256], "fft": [256, 256, 256], "dev": dev, "split": split}


def test_two_pass_bytes_are_the_fused_bytes_plus_one_extra_read_and_write_of_u():
    for s in (4, 8):
        fused = bench.alg_bytes("interp_precorr", s, _sizes(False))
        pre = bench.alg_bytes("interp_precorr", s, _sizes(True))
        st = bench.alg_bytes("interp_stencil", s, _sizes(True))
        assert pre + st == fused + 2 * s * 994_800


def test_precorrection_bytes_are_dominated_by_values_and_deltas():
    sz = _sizes(True)
    b32 = bench.alg_bytes("interp_precorr", 4, sz)
    b16 = bench.alg_bytes("interp_precorr", 4, sz, {"precorrection": 2})   # bfloat16 values
    nc = sz["dev"]["precorrection"]["entries"]
    assert b32 - b16 == 2 * nc
    assert 0.95 < nc * 6 / b32 < 1.0          # 4-byte values + 2-byte deltas are >95% of the bytes


def test_field_pass_reads_m_and_u_as_one_vector():
    sz = _sizes(True)
    Np, na = sz["Np"], sz["dev"]["adjacency"]["entries"]
    # row length + gradient and exchange values with deltas + (m, u) 4-vectors + RK4 stage state
    assert bench.alg_bytes("gradient_exchange", 4, sz) == 4 * Np + na * (2 + 16) + 16 * Np + 3.5 * 16 * Np


def test_bloch_pass_bytes_count_each_pass_once():
    # wire grid 128 x 128 x 256 with FFT 256^3: x passes 2 x (4.19M + 8.39M) complex values,
    # y passes 2 x (8.39M + 16.8M), z pass 2 x 16.8M complex and the 16.8M-value real spectrum
    n = bench.bloch_pass_bytes((128, 128, 256), (256, 256, 256), 4)
    assert n == 939_524_096
    assert bench.bloch_pass_bytes((128, 128, 256), (256, 256, 256), 8) == 2 * n
    # a fully periodic grid (no padding): each of the five passes reads and writes the whole grid
    # once (8 B per complex value), and the z pass reads the spectrum (4 B per point)
    assert bench.bloch_pass_bytes((8, 8, 8), (8, 8, 8), 4) == 512 * (5 * 2 * 8 + 4)
