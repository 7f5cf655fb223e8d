"""The split-bfloat16 tcgen05 GEMM (k_tc_gemm) and its persistent schedule, through mlcc_gemm.

One CTA per SM runs whole waves of 128 x 256 tiles data-parallel and the remaining tiles
stream-K: their K blocks are cut into equal ranges, one per CTA, and a tile that several
CTAs share is summed from their fp32 partials. Integer operands with |a|, |b| <= 15 are
exact in bfloat16 and every partial sum stays below 2^24, so the product is the exact
integer product whatever the schedule: a K block counted twice, a block left out or a
partial read from the wrong slot changes the result. The shapes hit each case of the
schedule on the device's SM count G: tiles a multiple of G (data-parallel only), one wave
and a remainder, two waves and a small remainder (few tiles shared by many CTAs), one wave
and a remainder of at least three quarters of a wave (data-parallel, last wave partial),
fewer tiles than SMs with long K (stream-K only), and a single tile with one K block.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BM, BN = 128, 256


@pytest.fixture(scope="module")
def ctx():
    from paper_2006_05226_gb300 import mlcc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mlcc.Context(0)
    yield c
    c.close()


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def _shape(case, G):
    """(M, N, K) for a schedule case, with ragged edges in M, N and K."""
    if case == "dp_only":        # tiles = G
        return BM * 2 - 5, BN * (G // 2) - 7, 640
    if case == "wave_and_rest":  # G < tiles < 2G
        return BM * 3 - 1, BN * ((4 * G) // 9) - 3, 1000
    if case == "waves_and_rest":  # tiles = 2G + 5
        return BM * 1 - 9, BN * (2 * G + 5) - 11, 1000
    if case == "wave_and_big_rest":  # tiles = G + 9G/10: the remainder runs data-parallel
        return BM * 1 - 9, BN * (G + (9 * G) // 10) - 11, 700
    if case == "few_tiles":      # 9 tiles, 33 K blocks: stream-K only, several CTAs per tile
        return 300, 520, 2100
    if case == "one_block":      # one tile, one K block
        return 17, 16, 64
    raise ValueError(case)


@pytest.mark.parametrize("case", ["dp_only", "wave_and_rest", "waves_and_rest", "wave_and_big_rest",
                                  "few_tiles", "one_block"])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, True)])
def test_integer_product_is_exact_under_every_schedule(ctx, case, ta, tb):
    from paper_2006_05226_gb300 import mlcc
    G = _sms()
    M, N, K = _shape(case, G)
    tiles = -(-M // BM) * -(-N // BN)
    if case == "dp_only":
        assert tiles % G == 0
    elif case == "wave_and_rest":
        assert G < tiles < 2 * G
    elif case == "waves_and_rest":
        assert tiles > 2 * G and tiles % G != 0
    elif case == "wave_and_big_rest":
        assert G < tiles < 2 * G and 4 * (tiles - G) >= 3 * G
    rng = np.random.default_rng(hash((case, ta, tb)) % 2 ** 32)
    A = rng.integers(-15, 16, size=(M, K)).astype(np.float64)
    B = rng.integers(-15, 16, size=(K, N)).astype(np.float64)
    C0 = rng.integers(-1000, 1000, size=(M, N)).astype(np.float64)
    dA = torch.as_tensor(np.ascontiguousarray(A.T if ta else A), device="cuda")
    dB = torch.as_tensor(np.ascontiguousarray(B.T if tb else B), device="cuda")
    dC = torch.as_tensor(C0, device="cuda")
    ctx.gemm(dA, dB, dC, alpha=2.0, beta=-1.0, trans_a=ta, trans_b=tb, precision=mlcc.MLCC_BF16)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    want = 2.0 * (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64) - C0
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} wrong elements, first at {bad[0].tolist()}: {got[tuple(bad[0])]} vs {want[tuple(bad[0])]}"


def test_split_product_accuracy_and_repeatability(ctx):
    """BF16X3 on random binary64 operands: within the split's bound of numpy's product, and
    bit-identical on a second call (the stream-K partials are added in a fixed order)."""
    from paper_2006_05226_gb300 import mlcc
    G = _sms()
    M, N, K = BM * 3 - 1, BN * ((4 * G) // 9) - 3, 3000
    rng = np.random.default_rng(5)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    dA = torch.as_tensor(A, device="cuda")
    dB = torch.as_tensor(B, device="cuda")
    out = []
    for _ in range(2):
        dC = torch.zeros((M, N), dtype=torch.float64, device="cuda")
        ctx.gemm(dA, dB, dC, precision=mlcc.MLCC_BF16X3)
        torch.cuda.synchronize()
        out.append(dC.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    want = A @ B
    bound = 2.0 ** -15 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(out[0] - want) <= bound)
