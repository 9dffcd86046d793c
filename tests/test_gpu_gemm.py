"""The tensor-core BF16 GEMM (warplda_gemm_bf16, tcgen05) against an FP64
product of the same BF16 values computed on the host."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    t.cuda.set_device(0)
    from paper_1510_08628_gb300 import warplda
    warplda.load()
    return t


# shapes with one CTA per tile (128 x 128 x 64) and with K split over 2 to 8
# CTAs (the encoder's forward 256 x 1024 x 512 and backward 256 x 512 x 1024,
# 1024 x 512 x 256 products among them)
@pytest.mark.parametrize("M,N,K,bias", [(128, 128, 64, False), (128, 256, 128, True),
                                        (384, 128, 512, False), (256, 1024, 512, True),
                                        (512, 512, 1024, True), (256, 512, 1024, False),
                                        (1024, 512, 256, False)])
def test_gemm_matches_fp64(torch, M, N, K, bias):
    from paper_1510_08628_gb300 import warplda
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    b = torch.randn(N, generator=g) if bias else None
    C = torch.empty(M, N, dtype=torch.float32, device="cuda")
    warplda.gemm_bf16(A.cuda(), B.cuda(), C, b.cuda() if bias else None)
    torch.cuda.synchronize()
    want = A.double().numpy() @ B.double().numpy().T
    if bias:
        want = want + b.double().numpy()[None, :]
    got = C.cpu().double().numpy()
    err = np.abs(got - want).max()
    assert err <= 1e-5 * np.abs(want).max() * np.sqrt(K), (err, np.abs(want).max())


def test_gemm_split_k_is_deterministic(torch):
    """The split-K partial tiles are added in a fixed order: repeated
    products are bit-identical."""
    from paper_1510_08628_gb300 import warplda
    g = torch.Generator().manual_seed(5)
    A = torch.randn(256, 1024, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(512, 1024, generator=g).to(torch.bfloat16).cuda()
    outs = []
    for _ in range(3):
        C = torch.empty(256, 512, dtype=torch.float32, device="cuda")
        warplda.gemm_bf16(A, B, C, None)
        torch.cuda.synchronize()
        outs.append(C.cpu())
    assert all(torch.equal(outs[0], o) for o in outs[1:])


def test_gemm_rejects_bad_shapes(torch):
    from paper_1510_08628_gb300 import warplda
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(100, 128, dtype=torch.float32, device="cuda")
    with pytest.raises(warplda.WarpLDAError):
        warplda.gemm_bf16(A, B, C)
