"""The tcgen05 tensor-core contraction on its own (through the C ABI diagnostics
entry), against plain products of the same operands.

Tolerances: one BF16 term is compared with the FP64 product of the BF16-rounded
operands (rounded directly from FP64, ties to even, as the kernel's split does) (only the FP32 accumulation differs: <= 1e-5 of sum |a||b|); three
terms (hi/lo splits) with the FP64 product of the unrounded operands
(<= 4e-5 of sum |a||b|: each operand keeps ~16 significant bits).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
bnb = pytest.importorskip("paper_2602_04551_b300")

def _bf16(x):
    """Round float64 to the nearest BF16 value (ties to even), directly from float64."""
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


CASES = [
    # M, N, Kd, nsplit, bn, splits
    (128, 128, 64, 1, 128, 1),
    (256, 128, 512, 1, 128, 1),
    (200, 100, 1000, 1, 128, 1),      # ragged M, N and K tails
    (200, 300, 1000, 1, 256, 3),      # split-K, two N tiles
    (256, 256, 640, 3, 128, 1),
    (333, 77, 1111, 3, 128, 4),
    (128, 512, 4096, 3, 256, 2),
    (200, 300, 1000, 2, 256, 3),      # 2 terms: A one BF16 term, B a pair
    (333, 77, 1111, 2, 128, 1),
]


@pytest.mark.parametrize("M,N,Kd,nsplit,bn,splits", CASES)
def test_tc_gemm_matches_plain_product(M, N, Kd, nsplit, bn, splits):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 13 + Kd)
    A = torch.randn(M, Kd, generator=g, dtype=torch.float64)
    B = torch.randn(N, Kd, generator=g, dtype=torch.float64)
    dA, dB = A.cuda(), B.cuda()
    dC = torch.empty(N, M, dtype=torch.float32, device="cuda")   # M x N column-major
    err = bnb.bnb_tc_gemm_check(dA, dB, M, N, Kd, nsplit, bn, splits, dC)
    assert err == 0
    _compare(A, B, dC.cpu().double().T.numpy(), nsplit)


CLUSTER_CASES = [
    # M, N, Kd, nsplit, cluster
    (128, 256, 64, 1, 1),             # one CTA, one K step
    (1000, 512, 5000, 3, 8),          # the X W'^T shape of a n=1000, p=5000, K=512 batch
    (1000, 512, 1000, 3, 8),          # the G^-1 T shape (two K steps per CTA)
    (300, 100, 1111, 3, 3),           # ragged M, N, K; cluster size not a power of two
    (129, 300, 200, 1, 8),            # more CTAs asked for than K steps: 4 chunks
    (257, 513, 777, 3, 2),
    (1000, 512, 5000, 2, 4),          # 2 terms, the X W'^T shape
    (300, 100, 1111, 2, 3),
]


@pytest.mark.parametrize("M,N,Kd,nsplit,cluster", CLUSTER_CASES)
def test_tc_gemm_cluster_matches_plain_product(M, N, Kd, nsplit, cluster):
    g = torch.Generator(device="cpu").manual_seed(M * 5 + N * 11 + Kd + cluster)
    A = torch.randn(M, Kd, generator=g, dtype=torch.float64)
    B = torch.randn(N, Kd, generator=g, dtype=torch.float64)
    dC = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    err = bnb.bnb_tc_gemm_check_cluster(A.cuda(), B.cuda(), M, N, Kd, nsplit, cluster, dC)
    assert err == 0
    _compare(A, B, dC.cpu().double().T.numpy(), nsplit)


def test_tc_gemm_cluster_is_deterministic():
    g = torch.Generator(device="cpu").manual_seed(3)
    A = torch.randn(1000, 3000, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(512, 3000, generator=g, dtype=torch.float64).cuda()
    outs = []
    for _ in range(3):
        dC = torch.empty(512, 1000, dtype=torch.float32, device="cuda")
        assert bnb.bnb_tc_gemm_check_cluster(A, B, 1000, 512, 3000, 3, 8, dC) == 0
        outs.append(dC.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


PAIR_CASES = [
    # M, N, Kd, nsplit, bn
    (256, 144, 64, 1, 144),           # one pair tile, one K step
    (512, 5000, 1000, 3, 144),        # (X^T U')^T of a n=1000, p=5000, K=512 batch
    (300, 333, 777, 3, 128),          # ragged rows (second tile partial), columns and K
    (200, 100, 1000, 2, 144),         # 2 terms: A the pair, B one BF16 term
    (1000, 700, 500, 1, 256),         # one accumulator of 256 columns
    (2048, 5000, 256, 3, 128),        # 320 tiles: several per pair, both accumulators
    (4096, 2000, 128, 1, 256),        # 128 tiles on single-accumulator pairs
]


@pytest.mark.parametrize("M,N,Kd,nsplit,bn", PAIR_CASES)
def test_tc_gemm_pair_matches_plain_product(M, N, Kd, nsplit, bn):
    g = torch.Generator(device="cpu").manual_seed(M * 3 + N * 17 + Kd + bn)
    A = torch.randn(M, Kd, generator=g, dtype=torch.float64)
    B = torch.randn(N, Kd, generator=g, dtype=torch.float64)
    dC = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    err = bnb.bnb_tc_gemm_check_pair(A.cuda(), B.cuda(), M, N, Kd, nsplit, bn, dC)
    assert err == 0
    C = dC.cpu().double().T.numpy()
    if nsplit == 2:   # in the pair kernel the first operand is the hi/lo pair
        _compare(B, A, C.T, nsplit)
    else:
        _compare(A, B, C, nsplit)


def test_tc_gemm_pair_is_deterministic():
    g = torch.Generator(device="cpu").manual_seed(5)
    A = torch.randn(512, 1000, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(5000, 1000, generator=g, dtype=torch.float64).cuda()
    outs = []
    for _ in range(3):
        dC = torch.empty(5000, 512, dtype=torch.float32, device="cuda")
        assert bnb.bnb_tc_gemm_check_pair(A, B, 512, 5000, 1000, 3, 144, dC) == 0
        outs.append(dC.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def _compare(A, B, C, nsplit):
    if nsplit == 2:
        # A rounded to one BF16 term (ties to even), B kept to ~16 bits by its pair
        Ar = torch.from_numpy(_bf16(A.numpy()))
        ref = (Ar @ B.T).numpy()
        scale = (Ar.abs() @ B.abs().T).numpy()
        assert np.all(np.abs(C - ref) <= 4e-5 * scale + 1e-6), np.max(np.abs(C - ref) / (scale + 1e-30))
        return
    if nsplit == 1:
        Ar = torch.from_numpy(_bf16(A.numpy()))
        Br = torch.from_numpy(_bf16(B.numpy()))
        ref = (Ar @ Br.T).numpy()
        scale = (Ar.abs() @ Br.abs().T).numpy()
        tol = 1e-5
    else:
        ref = (A @ B.T).numpy()
        scale = (A.abs() @ B.abs().T).numpy()
        tol = 4e-5
    assert np.all(np.abs(C - ref) <= tol * scale + 1e-6), np.max(np.abs(C - ref) / (scale + 1e-30))


@pytest.mark.parametrize("ctas,stages,b_rows", [(120, 3, 88), (148, 3, 88), (30, 4, 64)])
def test_tma_operand_ring_streams_every_stage(ctas, stages, b_rows):
    """The TMA operand ring alone (the fused product's stage: A hi/lo 128 rows, B hi/lo
    b_rows rows) on up to every SM: every bounded wait completes, the bytes delivered are
    the stage bytes of every pass, and the rate per SM is a plausible figure."""
    r = bnb.bnb_diag_tma_stream(ctas, stages, b_rows, reps=4, launches=3)
    assert r["err"] == 0, r
    stage = 2 * 128 * 64 * 2 + 2 * b_rows * 64 * 2
    assert r["bytes"] == ctas * 4 * 16 * stage
    assert 5.0 < r["gbs_per_sm"] < 2000.0, r
