"""The BF16 rounding the precision form applies to the positions, on the CPU.

The BF16 form's GPU parity tests compare its epochs with the oracle's FP64
epoch on the BF16-rounded positions (and separately on the FP32 ones); this
file pins the rounding helper they use and the size of the error the
rounding alone causes, measured with the oracle on both sets of positions.
"""
import numpy as np
import pytest

from conftest import bf16_round


def test_bf16_round_is_round_to_nearest_even():
    """bf16_round against torch's float32 -> bfloat16 conversion (round to
    nearest, ties to even) on random values of many magnitudes, on exact
    ties (the low 16 bits 0x8000, with an even and an odd kept part) and on
    values next to them."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = (rng.normal(size=20000) * np.exp2(rng.integers(-40, 40, size=20000))).astype(np.float32)
    hi = rng.integers(0x0080, 0x7F00, size=4000, dtype=np.uint32) << 16
    ties = np.concatenate([hi | 0x8000, hi | 0x7FFF, hi | 0x8001, (hi | 0x8000) | 0x80000000]).view(np.float32)
    for v in (x, ties, np.array([0.0, -0.0, 1.0, -1.0, 3.0e38], np.float32)):
        want = torch.from_numpy(v.copy()).to(torch.bfloat16).float().numpy()
        np.testing.assert_array_equal(bf16_round(v).view(np.uint32), want.view(np.uint32))
    # ties go to the even neighbour: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == np.float32(1.0 + 2.0 ** -6)


def _err_rows(got, ref, floor):
    nr = np.linalg.norm(ref, axis=1)
    return np.linalg.norm(got - ref, axis=1) / np.maximum(np.maximum(nr, 1e-6 * nr.mean()), floor)


@pytest.mark.slow
def test_position_rounding_alone_sets_the_bf16_error_at_low_d(oracle_mod):
    """The oracle's FP64 epoch on the BF16-rounded positions against its epoch
    on the FP32 positions (block sampling, the 120,000-vertex BA graph and
    the positions of the BF16 form's GPU tests): at d = 16 and sigma = 2 the
    rounding alone moves the worst vertex's step by more than the 1e-2 bar
    (about 4e-2: each distance sums the rounding of only 16 coordinates),
    at d = 64 by well under it."""
    from paper_2011_03479_gb300 import inputs
    rp, ci = inputs.barabasi_albert(120000, 8, seed=3102)
    n = len(rp) - 1
    worst = {}
    for d, sigma in [(16, 2.0), (64, 0.7)]:
        x = (np.random.default_rng(8 + d).normal(size=(n, d)) * 0.7).astype(np.float32)
        xb = bf16_round(x).astype(np.float64)
        kw = dict(block_partners=64, tile_vertices=128)
        ref = oracle_mod.epoch(rp, ci, x.astype(np.float64), sigma, 9, 0x6E6D7065, 5, **kw)
        emu = oracle_mod.epoch(rp, ci, xb, sigma, 9, 0x6E6D7065, 5, **kw)
        np.testing.assert_array_equal(emu["partners"], ref["partners"])   # samples do not see positions
        step_ref = ref["x_new"] - x.astype(np.float64)
        step_emu = emu["x_new"] - xb
        e_x = _err_rows(step_emu, step_ref, 3e-2 * ref["abs_terms"] / ref["z"])
        worst[d] = float(e_x.max())
    print(f"step moved by the rounding alone: d=16 {worst[16]:.2e}, d=64 {worst[64]:.2e}")
    assert worst[16] > 2e-2
    assert worst[64] < 5e-3
