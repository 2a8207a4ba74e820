"""The tcgen05 BF16 GEMM against a plain PyTorch FP32 reference of the same
op (BF16-rounded inputs, FP32 products), with every epilogue (needs a
GB300)."""
import ctypes

import pytest

from paper_2601_01903_gb300 import native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _gemm(A, B, bias=None, act=0, dz=None, want=("f",)):
    lib = native.load()
    M, K = A.shape
    N = B.shape[0]
    Cf = torch.full((M, N), float("nan"), device="cuda") if "f" in want else None
    Cb = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda") if "b" in want else None
    Ct = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda") if "t" in want else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.tt_fsi_gemm_bf16(_p(A), A.stride(0), _p(B), B.stride(0), M, N, K, _p(bias), act, _p(dz),
                              N, _p(Cf), N, _p(Cb), N, _p(Ct), M, _p(err),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return Cf, Cb, Ct


def _ref(A, B):
    return A.float() @ B.float().T


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 128, 16), (200, 137, 144), (384, 256, 1024),
                                   (4096, 1024, 1024), (4096, 144, 1024), (1024, 16, 4096), (1, 8, 8),
                                   (257, 129, 80)])
def test_gemm_matches_fp32_reference(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    Cf, _, _ = _gemm(A, B)
    ref = _ref(A, B)
    assert torch.allclose(Cf, ref, rtol=1e-4, atol=1e-3 * K ** 0.5), (Cf - ref).abs().max().item()


def test_gemm_epilogues():
    g = torch.Generator(device="cuda").manual_seed(5)
    M, N, K = 300, 200, 96
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    z = _ref(A, B) + bias
    Cf, Cb, Ct = _gemm(A, B, bias=bias, act=1, want=("f", "b", "t"))
    assert torch.allclose(Cf, z, rtol=1e-4, atol=1e-3)
    gel = torch.nn.functional.gelu(z)
    assert torch.allclose(Cb.float(), gel, rtol=1e-2, atol=1e-2)
    assert torch.equal(Ct, Cb.T.contiguous())
    dz = torch.randn(M, N, device="cuda", generator=g)
    Cf2, Cb2, _ = _gemm(A, B, dz=dz, want=("f", "b"))
    zz = dz.clone().requires_grad_(True)
    (torch.nn.functional.gelu(zz) * _ref(A, B)).sum().backward()
    assert torch.allclose(Cf2, zz.grad, rtol=1e-4, atol=1e-3)
