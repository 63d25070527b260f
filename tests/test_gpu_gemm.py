"""The DeepONet trunk's GEMMs (Sec. 2.4) on the tensor cores, through the
C ABI test hook, against FP64 products of the same operands.

Two forms run on tcgen05: the pixel GEMM (the trunk's layers and their data
gradients: pixels the long N dimension) and the reduction GEMM (the weight
gradients: pixels the K dimension).  The tensor cores take TF32 operands;
the kernels split every operand into a TF32 high part and an FP32
remainder and add hi hi + hi lo + lo hi, so a product is FP32-accurate
(the dropped lo lo term is 2^-20 of it).  The bar is 5e-5 * sum_k |A(m,k)
B(k,n)| per entry, the FP32 accumulation of up to 8,192 products (plain
TF32 operands are off by up to ~1e-3 of that sum, a transposed operand, a
dropped bias or a wrong tile by O(1)).  The CUDA-core kernel meets 1e-5.
Shapes are ragged: pixel counts that end in a partial tile, channel counts
that are not multiples of the MMA sizes."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01800_gb300 import _lib
    return _lib


def _run(lib, M, N, K, transA, transB, bias, act, accumulate, impl, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((K, M) if transA else (M, K)).astype(np.float32)
    B = g.standard_normal((N, K) if transB else (K, N)).astype(np.float32)
    C0 = g.standard_normal((M, N)).astype(np.float32)
    bv = g.standard_normal(M).astype(np.float32) if bias else None
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    Cd = torch.tensor(C0, device="cuda")
    bd = torch.tensor(bv, device="cuda") if bias else None
    form = ctypes.c_int(-1)
    st = lib.load().ppe_debug_gemm(M, N, K, ctypes.c_void_p(Ad.data_ptr()), A.shape[1], int(transA),
                                   ctypes.c_void_p(Bd.data_ptr()), B.shape[1], int(transB),
                                   ctypes.c_void_p(Cd.data_ptr()), N,
                                   ctypes.c_void_p(bd.data_ptr()) if bias else None, act, int(accumulate), impl,
                                   ctypes.byref(form), None)
    lib.check(st, "ppe_debug_gemm")
    torch.cuda.synchronize()
    Am = (A.T if transA else A).astype(np.float64)
    Bm = (B.T if transB else B).astype(np.float64)
    z = Am @ Bm + (bv.astype(np.float64)[:, None] if bias else 0.0)
    y = np.tanh(z) if act == 1 else z
    ref = y + (C0 if accumulate else 0.0)
    scale = np.abs(Am) @ np.abs(Bm) + (np.abs(bv)[:, None] if bias else 0.0)
    return Cd.cpu().numpy().astype(np.float64), ref, scale, form.value


PIXEL = [  # M, N (pixels), K, transA, bias, act, accumulate
    (200, 3000, 100, False, True, 1, False),     # trunk layer 2 -> hidden 200, tanh; ragged last tile
    (100, 2048, 200, False, True, 0, False),     # trunk layer 3
    (32, 1500, 100, True, False, 0, False),      # head fold (transposed weights)
    (100, 1100, 32, False, False, 0, True),      # head data gradient, accumulated
    (200, 1024, 100, True, False, 0, False),     # transposed-weight data gradient
    (17, 1301, 9, False, True, 1, False),        # odd sizes: one 8-channel step
    (1, 1500, 100, False, True, 0, False),       # one output channel (the head's bias fold)
]

REDUCTION = [  # M, N, K (pixels), accumulate
    (100, 200, 5000, False),                     # ragged pixel chunk
    (200, 100, 8192, False),                     # two M blocks of 128
    (100, 32, 4096, True),
    (19, 23, 4100, False),
]


@pytest.mark.parametrize("M,N,K,transA,bias,act,acc", PIXEL)
def test_pixel_gemm_tensor_cores(lib, M, N, K, transA, bias, act, acc):
    C, ref, scale, form = _run(lib, M, N, K, transA, False, bias, act, acc, 0, M + N + K)
    assert form == 1
    err = np.abs(C - ref)
    assert np.all(err <= 5e-5 * scale + 1e-6), (err.max(), np.max(err / (scale + 1e-30)))


@pytest.mark.parametrize("M,N,K,acc", REDUCTION)
def test_reduction_gemm_tensor_cores(lib, M, N, K, acc):
    C, ref, scale, form = _run(lib, M, N, K, False, True, False, 0, acc, 0, M * N + K)
    assert form == 2
    err = np.abs(C - ref)
    assert np.all(err <= 5e-5 * scale + 1e-6), (err.max(), np.max(err / (scale + 1e-30)))


def test_reduction_gemm_is_deterministic(lib):
    a = _run(lib, 100, 200, 6000, False, True, False, 0, False, 0, 5)[0]
    b = _run(lib, 100, 200, 6000, False, True, False, 0, False, 0, 5)[0]
    assert np.array_equal(a, b)


THIN = [  # M, N, K, transA, transB, bias, act, accumulate, form
    (100, 2, 8192, False, True, False, 0, False, 3),     # first layer's weight gradient (2 coordinates)
    (100, 1, 5003, False, False, False, 0, True, 3),     # a bias gradient against a vector, accumulated
    (1, 1, 4099, False, False, False, 0, False, 3),      # the output bias's gradient
    (100, 1200, 2, False, False, True, 1, False, 4),     # first trunk layer: tanh(W xy + b)
    (37, 1500, 1, False, False, False, 0, True, 4),      # rank-one term, accumulated
    (300, 1500, 100, False, False, False, 0, False, 0),  # outside every special form
]


@pytest.mark.parametrize("M,N,K,transA,transB,bias,act,acc,want", THIN)
def test_thin_forms(lib, M, N, K, transA, transB, bias, act, acc, want):
    """The thin products run on the CUDA cores (row dots, small K) at FP32
    accuracy."""
    C, ref, scale, form = _run(lib, M, N, K, transA, transB, bias, act, acc, 0, 11 + M + K)
    assert form == want
    assert np.all(np.abs(C - ref) <= 1e-5 * scale + 1e-6)


@pytest.mark.parametrize("M,N,K,transA,bias,act,acc", PIXEL[:3])
def test_cuda_core_kernel(lib, M, N, K, transA, bias, act, acc):
    C, ref, scale, form = _run(lib, M, N, K, transA, False, bias, act, acc, 1, 7)
    assert form == 0
    assert np.all(np.abs(C - ref) <= 1e-5 * scale + 1e-6)
