"""The tcgen05 bf16 GEMM (surrogate building block) against an fp32 matmul of
the same bf16 operands, for every fused epilogue, tile width, ragged M and N
(the element-wise tail path) and the transposed copy of the training step;
the one-CTA and pair-CTA (cta_group::2) kernels on the same shapes; the GELU
and GELU' epilogues against the correctly rounded bf16 of the exact function."""
import math

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
    """GELU, erf form, in fp64."""
    z = z.double()
    return 0.5 * z * (1 + torch.erf(z / 2 ** 0.5))


def operands(M, N, K, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = (torch.randn(M, K, generator=g) / K ** 0.5).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).cuda()
    return A, B, bias


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 256, 1024), (256, 1024, 1024), (130, 128, 192),
                                   (512, 64, 256), (1000, 4096, 128), (257, 200, 128), (70, 96, 64)])
@pytest.mark.parametrize("with_bias", [True, False])
def test_gemm_f32_epilogue(M, N, K, with_bias):
    A, B, bias = operands(M, N, K, M + N + K)
    if not with_bias:
        bias = None
    out = torch.empty(M, N, device="cuda")
    abi.tmm_gemm_bf16(A, B, bias, 0, out)
    ref = A.float() @ B.float().T + (bias if bias is not None else 0.0)
    err = (out - ref).abs().max().item()
    assert err <= 1e-4 * max(1.0, ref.abs().max().item()), err


def check_gelu(M, N, K, seed):
    A, B, bias = operands(M, N, K, seed)
    z = A.float() @ B.float().T + bias
    out = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    aux = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    ldoT = (M + 7) // 8 * 8 + 8
    outT = torch.full((N, ldoT), 7.0, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16_t(A, B, bias, 1, out, aux, outT)
    # pre-activation: bf16 of the fp32 accumulator
    assert (aux.float() - z).abs().max().item() <= 4e-3 * max(1.0, z.abs().max().item())
    # activation: bf16 of GELU(aux), within bf16 rounding of the fp64 value
    ref = ref_gelu(aux.float())
    dev = (out.double() - ref).abs() - (4e-3 * ref.abs() + 2e-6 * (aux.double().abs() + 1))
    assert dev.max().item() <= 0, dev.max().item()
    # transposed copy: the same bits, columns past M untouched
    assert torch.equal(outT[:, :M], out.T)
    assert bool((outT[:, M:] == 7.0).all())
    # derivative epilogue reads the saved pre-activation
    out2 = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    out2T = torch.full((N, ldoT), 7.0, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16_t(A, B, None, 2, out2, aux, out2T)
    zz = aux.double().requires_grad_(True)
    ref_gelu(zz).sum().backward()
    ref2 = (A.float() @ B.float().T).double() * zz.grad
    tol = 4e-3 * ref2.abs() + 1e-4 * max(1.0, ref2.abs().max().item())
    assert bool(((out2.double() - ref2).abs() <= tol).all())
    assert torch.equal(out2T[:, :M], out2.T)
    assert bool((out2T[:, M:] == 7.0).all())
    # clamp epilogue
    out3 = torch.empty(M, N, device="cuda")
    abi.tmm_gemm_bf16(A, B, bias, 3, out3)
    assert (out3 - z.clamp(0, 1)).abs().max().item() <= 1e-4 * max(1.0, z.abs().max().item())


@pytest.mark.parametrize("M,N,K", [(384, 256, 512), (300, 1024, 256), (97, 200, 64), (640, 64, 128)])
def test_gemm_gelu_dgelu_transpose_and_clamp(M, N, K):
    check_gelu(M, N, K, M * 7 + N)


def test_gemm_gelu_without_transposed_copy_matches():
    M, N, K = 256, 512, 256
    A, B, bias = operands(M, N, K, 11)
    out = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    aux = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16(A, B, bias, 1, out, aux)
    out_t = torch.empty_like(out)
    aux_t = torch.empty_like(aux)
    outT = torch.empty(N, M, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16_t(A, B, bias, 1, out_t, aux_t, outT)
    assert torch.equal(out, out_t) and torch.equal(aux, aux_t) and torch.equal(outT, out.T)


def test_gemm_transposed_entry_rejects_bad_arguments():
    A, B, bias = operands(64, 64, 64, 1)
    out = torch.empty(64, 64, dtype=torch.bfloat16, device="cuda")
    outT = torch.empty(64, 32, dtype=torch.bfloat16, device="cuda")  # ldoT < M
    with pytest.raises(RuntimeError):
        abi.tmm_gemm_bf16_t(A, B, bias, 1, out, None, outT)
    outT = torch.empty(64, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(RuntimeError):
        abi.tmm_gemm_bf16_t(A, B, bias, 0, torch.empty(64, 64, device="cuda"), None, outT)


FORMS = ["single", "pair"]


@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 1024, 256), (1000, 512, 192), (4096, 1024, 1024),
                                   (130, 256, 64), (100, 512, 128), (513, 300, 64)])
def test_pair_and_single_forms_agree_bit_for_bit(M, N, K, monkeypatch):
    A, B, bias = operands(M, N, K, M + 3 * N)
    outs = []
    for form in FORMS:
        monkeypatch.setenv("TMM_GEMM_FORM", form)
        o32 = torch.empty(M, N, device="cuda")
        abi.tmm_gemm_bf16(A, B, bias, 0, o32)
        ob = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
        aux = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
        abi.tmm_gemm_bf16(A, B, bias, 1, ob, aux)
        od = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
        abi.tmm_gemm_bf16(A, B, None, 2, od, aux)
        outs.append((o32, ob, aux, od))
    ref = A.float() @ B.float().T + bias
    assert (outs[0][0] - ref).abs().max().item() <= 1e-4 * max(1.0, ref.abs().max().item())
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def _bf16_ulp(x):
    """One bf16 unit in the last place of |x| (x != 0), as float64."""
    e = torch.floor(torch.log2(x.abs()))
    return torch.pow(2.0, e - 7)


@pytest.mark.parametrize("form", FORMS)
def test_gelu_epilogues_round_the_exact_function(form, monkeypatch):
    """B = I passes each bf16 z of A through the accumulator exactly, so the
    GELU epilogue's output is its bf16 of GELU(z) and the GELU' epilogue's (with
    A = 1) its bf16 of GELU'(aux).  Against the exact functions (fp64, erfc form,
    accurate in both tails): within one bf16 unit everywhere, and the correctly
    rounded value for all but near-ties."""
    monkeypatch.setenv("TMM_GEMM_FORM", form)
    M, N = 2048, 256
    z = torch.linspace(-12.0, 12.0, M * N, dtype=torch.float64)
    z = z[torch.randperm(M * N, generator=torch.Generator().manual_seed(3))].reshape(M, N)
    zb = z.to(torch.bfloat16)
    eye = torch.eye(N, dtype=torch.bfloat16, device="cuda")
    out = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    aux = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16(zb.cuda(), eye, None, 1, out, aux)
    assert torch.equal(aux.cpu(), zb)
    x = zb.double()
    g = 0.5 * x * torch.special.erfc(-x / math.sqrt(2.0))
    dg = 0.5 * torch.special.erfc(-x / math.sqrt(2.0)) + x * torch.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    ones = torch.ones(M, N, dtype=torch.bfloat16, device="cuda")
    dout = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    abi.tmm_gemm_bf16(ones, eye, None, 2, dout, aux)
    for got, ref in ((out.cpu().double(), g), (dout.cpu().double(), dg)):
        nz = ref != 0
        assert bool(((got - ref).abs()[nz] <= _bf16_ulp(ref[nz])).all())
        exact = (got == ref.to(torch.bfloat16).double()).double().mean().item()
        assert exact >= 0.999, exact
