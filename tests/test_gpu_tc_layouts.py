"""Pins of the tensor-core conventions the fused kernel is built on.

One tcgen05 MMA on integer data (exact in FP32) per case: K-major and
MN-major shared-memory operands with SWIZZLE_NONE descriptors, A in tensor
memory, and the row -> TMEM lane layout of M = 128 and M = 64 results.
"""
import numpy as np
import pytest

from paper_2207_11669_gb300 import dcf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_11669_gb300 import build
    build.build()


def ref(M, N, K):
    i = np.arange(M, dtype=np.uint64)[:, None]
    k = np.arange(K, dtype=np.uint64)[None, :]
    m32 = np.uint64(0xFFFFFFFF)
    ha = ((i * np.uint64(2654435761)) & m32) ^ ((k * np.uint64(40503)) & m32)
    A = ((ha >> np.uint64(13)) % np.uint64(9)).astype(np.float64) - 4
    j = np.arange(N, dtype=np.uint64)[:, None]
    hb = ((j * np.uint64(2246822519)) & m32) ^ ((k * np.uint64(3266489917)) & m32)
    B = ((hb >> np.uint64(15)) % np.uint64(7)).astype(np.float64) - 3
    return A @ B.T


def lanes_m64(D, expected):
    """Which TMEM lane holds each of the 64 result rows (-1 if none)."""
    where = []
    for row in range(expected.shape[0]):
        hits = [l for l in range(128) if np.array_equal(D[l, :expected.shape[1]], expected[row])]
        where.append(hits[0] if hits else -1)
    return where


CASES = {
    # name: cfg = M, N, K, a_kind, a_lbo, a_sbo, dA_lbo, dA_sbo, b_lbo, b_sbo, dB_lbo, dB_sbo
    "kmajor_m128": [128, 64, 32, 0, 128, 512, 128, 512, 128, 512, 128, 512],
    "kmajor_m128_mcontig": [128, 64, 32, 0, 2048, 128, 2048, 128, 1024, 128, 1024, 128],
    "mnmajor_m128": [128, 64, 32, 1, 128, 512, 128, 512, 128, 512, 128, 512],
    "mnmajor_m64": [64, 64, 32, 1, 128, 512, 128, 512, 128, 512, 128, 512],
    "tmem_a_m128": [128, 32, 32, 2, 128, 512, 128, 512, 128, 512, 128, 512],
}


def diagnose(cfg, D, exp):
    """Describe a mismatch: which alternative reading of the layout matches."""
    notes = [f"max abs diff {np.max(np.abs(D[:128, :cfg[1]] - exp)):.1f}"]
    if np.array_equal(D[:128, :cfg[1]], exp.T[:128, :cfg[1]] if exp.shape[0] == exp.shape[1] else exp):
        notes.append("matches transposed")
    alt = list(cfg)
    alt[6], alt[7] = cfg[7], cfg[6]          # swap LBO/SBO in A's descriptor
    try:
        D2 = dcf.dcf_tc_selftest(alt)
        notes.append(f"swapped A desc matches: {np.array_equal(D2[:128, :cfg[1]], exp)}")
    except dcf.DcfError as e:
        notes.append(f"swapped A desc: {e}")
    return "; ".join(notes)


@pytest.mark.parametrize("name", ["kmajor_m128", "kmajor_m128_mcontig", "mnmajor_m128",
                                  "tmem_a_m128"])
def test_m128_rows_in_lanes(name):
    cfg = CASES[name]
    D = dcf.dcf_tc_selftest(cfg)
    exp = ref(cfg[0], cfg[1], cfg[2])
    ok = np.array_equal(D[:128, :cfg[1]], exp)
    assert ok, name + ": " + diagnose(cfg, D, exp)


def test_m64_result_layout():
    """M = 64: rows 16q .. 16q+15 sit in lanes 32q .. 32q+15."""
    cfg = CASES["mnmajor_m64"]
    D = dcf.dcf_tc_selftest(cfg)
    exp = ref(64, 64, 32)
    assert len({tuple(r) for r in exp}) == 64          # rows are distinguishable
    where = lanes_m64(D, exp)
    assert where == [32 * (r // 16) + r % 16 for r in range(64)], where
