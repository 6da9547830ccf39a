"""Tensor-core tile (tcgen05, BF16 x BF16 -> FP32) against a float64 CPU
matrix product of the same BF16 values: every majorness of A and B, ragged
M and N, every tile width, and the split-K path; and the bounded-wait timeout
path the tile's pipelines rely on."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1701_03549_gb300 import fire
    c = fire.fire_create(0, torch.cuda.current_stream())
    yield c
    c.close()


def _ref(A, B):
    a = A.double().cpu().numpy()
    b = B.double().cpu().numpy()
    return a @ b.T, np.abs(a) @ np.abs(b).T


@pytest.mark.parametrize("M,N,K,a_mn,b_mn,ksplit", [
    (128, 128, 64, False, False, 1),
    (300, 200, 192, False, False, 1),
    (128, 16, 64, False, False, 1),
    (257, 40, 128, False, False, 1),
    (130, 60, 256, False, False, 1),
    (256, 128, 128, True, False, 1),
    (136, 72, 192, False, True, 1),
    (128, 256, 512, True, True, 1),
    (1000, 128, 1024, False, False, 4),
    (128, 1152, 4096, True, True, 16),
])
def test_tc_gemm_matches_cpu(ctx, M, N, K, a_mn, b_mn, ksplit):
    from paper_1701_03549_gb300 import fire
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref, mag = _ref(A, B)
    Ad = (A.t().contiguous() if a_mn else A).cuda()
    Bd = (B.t().contiguous() if b_mn else B).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    torch.cuda.synchronize()
    fire.fire_tc_gemm(ctx, Ad, Bd, M, N, K, C, a_mn=a_mn, b_mn=b_mn,
                      ksplit=ksplit)
    got = C.cpu().double().numpy()
    assert np.isfinite(got).all()
    err = np.abs(got - ref)
    bound = 2.0 * K * 2.0 ** -24 * mag + 1e-30
    assert np.all(err <= bound), float((err / (mag + 1e-30)).max())


def test_tc_gemm_rejects_bad_shapes(ctx):
    from paper_1701_03549_gb300 import fire
    A = torch.zeros(128, 96, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 128, device="cuda")
    with pytest.raises(fire.FireError):
        fire.fire_tc_gemm(ctx, A, A, 128, 128, 96, C)      # K % 64 != 0
    A2 = torch.zeros(64, 132, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(fire.FireError):
        fire.fire_tc_gemm(ctx, A2, A2, 132, 128, 64, C, a_mn=True)  # M % 8


def test_bounded_wait_runs_out_and_the_context_survives(ctx):
    """The timeout path every TMA and tensor-core wait relies on: a wait on a
    barrier phase nothing completes gives up after about a second, the call
    reports FIRE_ETIMEOUT, and afterwards the error word is clear and the
    tensor-core tile still computes correct products."""
    import time

    from paper_1701_03549_gb300 import fire
    t0 = time.perf_counter()
    rc = fire.fire_wait_selftest(ctx)
    dt = time.perf_counter() - t0
    assert rc == fire.FIRE_ETIMEOUT
    assert 0.2 < dt < 30.0           # 2^31 SM clocks
    assert ctx.sync() == fire.FIRE_OK
    g = torch.Generator().manual_seed(5)
    A = torch.randn(128, 64, generator=g).to(torch.bfloat16)
    B = torch.randn(32, 64, generator=g).to(torch.bfloat16)
    C = torch.full((128, 32), float("nan"), device="cuda")
    fire.fire_tc_gemm(ctx, A.cuda(), B.cuda(), 128, 32, 64, C)
    want = A.double() @ B.double().t()
    assert torch.allclose(C.cpu().double(), want, rtol=0, atol=1e-4)
