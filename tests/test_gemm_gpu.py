"""The tcgen05 bf16 GEMM (surrogate building block) against an fp32 matmul of
the same bf16 operands, for every fused epilogue, tile width and a ragged M."""
import pytest
import torch

from paper_2111_13667_gb300 import abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def ref_gelu(z):
    return 0.5 * z * (1 + torch.erf(z / 2 ** 0.5))


def operands(M, N, K, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = (torch.randn(M, K, generator=g) / K ** 0.5).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).cuda()
    return A, B, bias


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 256, 1024), (256, 1024, 1024), (130, 128, 192),
                                   (512, 64, 256), (1000, 4096, 128)])
def test_gemm_f32_epilogue(M, N, K):
    A, B, bias = operands(M, N, K, M + N + K)
    out = torch.empty(M, N, device="cuda")
    abi.tmm_gemm_bf16(A, B, bias, 0, out)
    ref = A.float() @ B.float().T + bias
    err = (out - ref).abs().max().item()
    assert err <= 1e-4 * max(1.0, ref.abs().max().item()), err


def test_gemm_gelu_and_dgelu_and_clamp():
    M, N, K = 384, 256, 512
    A, B, bias = operands(M, N, K, 7)
    z = A.float() @ B.float().T + bias
    out = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    aux = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16(A, B, bias, 1, out, aux)
    assert (aux.float() - z).abs().max().item() <= 1e-2 * max(1.0, z.abs().max().item())
    assert (out.float() - ref_gelu(aux.float())).abs().max().item() <= 2e-2
    # derivative epilogue reads the saved pre-activation
    out2 = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16(A, B, None, 2, out2, aux)
    zz = aux.float().requires_grad_(True)
    ref_gelu(zz).sum().backward()
    ref2 = (A.float() @ B.float().T) * zz.grad
    assert (out2.float() - ref2).abs().max().item() <= 2e-2 * max(1.0, ref2.abs().max().item())
    out3 = torch.empty(M, N, device="cuda")
    abi.tmm_gemm_bf16(A, B, bias, 3, out3)
    assert (out3 - z.clamp(0, 1)).abs().max().item() <= 1e-4 * max(1.0, z.abs().max().item())
