"""cc_lr_selftest_gemm_noalloc: the tensor-core GEMM self-test run inside the library's fixed
device array, with no device allocation, against the allocating cc_lr_selftest_gemm.

Both compute the same products from the same seeded inputs.  Short products split K over
blocks whose partial sums are added with atomics, in an order that varies from run to run, so
the two agree within the tolerances of the GEMM self-test (tensor cores: 4e-3 for TF32,
1e-8 K + 2e-6 for 3xTF32; FP32 CUDA cores: 2e-5), not to the last bit.  The
entry point is called twice in a row, so the second call checks that the shared array is
cleared where it must be.  The file is named to be collected last: the first call on the
device does the set-up, and it must work both in a fresh process and after every other test.
"""
import math
import os
import subprocess
import sys

import pytest

from paper_2604_12914_gb300 import binding


def _order_tol(K):
    return 8.0 * math.sqrt(K) * 6e-8


def _tol(mode, K):
    # the tolerances of the tensor-core GEMM self-test in test_gpu_parity.py
    return 4e-3 if mode == 1 else 1e-8 * K + 2e-6


@pytest.mark.gpu
@pytest.mark.parametrize("M,N,K,mode", [(200, 136, 300, 1), (200, 136, 300, 2), (384, 384, 384, 2),
                                        (37, 5, 900, 2)])
def test_noalloc_matches_allocating_selftest(M, N, K, mode):
    tol = _tol(mode, K)
    # the no-allocation call comes first, so that in a fresh process it does its own set-up
    # before any other tensor-core work has run
    first = binding.cc_lr_selftest_gemm_noalloc(M, N, K, mode, seed=7)
    ref_tc, ref_fp32 = binding.cc_lr_selftest_gemm(M, N, K, mode, seed=7)
    assert 0 <= ref_tc < tol
    second = binding.cc_lr_selftest_gemm_noalloc(M, N, K, mode, seed=7)
    for call, (e_tc, e_fp32) in enumerate((first, second)):
        print(f"call {call}: M={M} N={N} K={K} mode={mode}: tc {e_tc:.3e} (allocating {ref_tc:.3e}) "
              f"fp32 {e_fp32:.3e} (allocating {ref_fp32:.3e})")
        assert 0 <= e_tc < tol
        assert 0 <= e_fp32 < 2e-5
        # the same products from the same inputs: only the order of the FP32 partial sums differs
        # (split K adds partial tiles with atomics), a few roundings times sqrt(K)
        assert abs(e_tc - ref_tc) <= _order_tol(K)
        assert abs(e_fp32 - ref_fp32) <= _order_tol(K)


def test_noalloc_rejects_sizes_beyond_the_array():
    """Checked before any device call, so it runs without a GPU as well."""
    with pytest.raises(RuntimeError, match="bytes of scratch"):
        binding.cc_lr_selftest_gemm_noalloc(512, 512, 512, 2)
    with pytest.raises(RuntimeError, match="bytes of scratch"):
        binding.cc_lr_selftest_gemm_noalloc(1 << 30, 1 << 30, 1 << 30, 1)


@pytest.mark.gpu
def test_noalloc_first_call_in_a_fresh_process():
    """In a new process the no-allocation entry point is the first library call, so its own
    set-up (the array's address, the tensor-map encoder, the kernel's shared-memory limit) runs
    there; its results equal the allocating self-test's in this process."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); from paper_2604_12914_gb300 import binding; "
            "print(*binding.cc_lr_selftest_gemm_noalloc(200, 136, 300, 2, seed=7))") % root
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    e_tc, e_fp32 = map(float, out.stdout.split()[-2:])
    ref_tc, ref_fp32 = binding.cc_lr_selftest_gemm(200, 136, 300, 2, seed=7)
    print(f"fresh process: tc {e_tc:.3e} fp32 {e_fp32:.3e}; allocating: tc {ref_tc:.3e} fp32 {ref_fp32:.3e}")
    assert 0 <= e_tc < _tol(2, 300)
    assert abs(e_tc - ref_tc) <= _order_tol(300)
    assert abs(e_fp32 - ref_fp32) <= _order_tol(300)
