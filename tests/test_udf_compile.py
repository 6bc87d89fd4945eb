"""Run-time compilation of user-defined integrands (CPU: NVRTC needs no GPU).

zmc_udf_create compiles the user's zmc_user_f together with the library's own
device code; these tests check the host side of that: good sources compile for
both precisions, a broken source is refused with the compiler's message, and the
arguments are validated.  The GPU tests (test_gpu_udf.py) run what is compiled.
"""
import ctypes

import pytest

from paper_2104_10073_gb300 import zmc


def _nvrtc_present() -> bool:
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            ctypes.CDLL(name)
            return True
        except OSError:
            pass
    return False


pytestmark = pytest.mark.skipif(not _nvrtc_present(), reason="NVRTC not installed")

F32_SRC = r"""
__device__ float zmc_user_f(const float *x, const float *p) {
  float r2 = 0.0f;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) r2 = fmaf(x[i] - p[1 + i], x[i] - p[1 + i], r2);
  return p[0] * expf(-r2);
}
"""

F64_SRC = r"""
__device__ double zmc_user_f(const double *x, const double *p) {
  double s = 0.0;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) s += p[i] * x[i] * x[i];
  return sqrt(1.0 + s);
}
"""


@pytest.mark.parametrize("dim", [1, 4, 7, 12])
def test_compiles_for_both_precisions(dim):
    a = zmc.Udf(F32_SRC, dim, zmc.ZMC_UDF_F32)
    b = zmc.Udf(F64_SRC, dim, zmc.ZMC_UDF_F64, amplitude=10.0)
    assert a.handle and b.handle
    assert isinstance(a.log, str)
    a.close()
    b.close()


def test_compile_error_is_reported():
    with pytest.raises(zmc.ZmcError) as e:
        zmc.Udf("__device__ float zmc_user_f(const float *x, const float *p) { return y; }", 3)
    assert e.value.status == zmc.ZMC_EINVAL
    assert "does not compile" in str(e.value) and "y" in str(e.value)


def test_missing_function_is_reported():
    with pytest.raises(zmc.ZmcError) as e:
        zmc.Udf("__device__ float other(float a) { return a; }", 2)
    assert e.value.status == zmc.ZMC_EINVAL


def test_wrong_precision_signature_is_reported():
    # a double form compiled as ZMC_UDF_F32: the float call does not match
    with pytest.raises(zmc.ZmcError) as e:
        zmc.Udf(F64_SRC.replace("const double *p", "const double *q").replace("p[i]", "q[i]"), 2,
                zmc.ZMC_UDF_F32)
    assert e.value.status == zmc.ZMC_EINVAL


@pytest.mark.parametrize("dim,prec,amp", [(0, 0, 0.0), (13, 0, 0.0), (2, 2, 0.0), (2, 0, -1.0),
                                          (2, 0, float("inf"))])
def test_arguments_are_validated(dim, prec, amp):
    with pytest.raises(zmc.ZmcError) as e:
        zmc.Udf(F32_SRC, dim, prec, amp)
    assert e.value.status == zmc.ZMC_EINVAL


HELPER_A = r"""
__device__ float helper(float v) { return v * v; }
__device__ float zmc_user_f(const float *x, const float *p) { return p[0] * helper(x[0]); }
"""
HELPER_B = r"""
__device__ float helper(float v) { return v + 1.0f; }
__device__ float zmc_user_f(const float *x, const float *p) {
  float s = 0.0f;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) s += helper(x[i]);
  return s;
}
"""


def test_multi_function_module_compiles_with_repeated_helper_names():
    u = zmc.Udf([HELPER_A, HELPER_B, F32_SRC], [1, 5, 3], zmc.ZMC_UDF_F32, [1.0, 10.0, 2.0])
    assert u.dims == [1, 5, 3]
    u.close()


def test_multi_function_error_names_the_source():
    with pytest.raises(zmc.ZmcError) as e:
        zmc.Udf([HELPER_A, "__device__ float zmc_user_f(const float *x, const float *p) "
                           "{ return undefined_name; }"], [1, 2])
    assert e.value.status == zmc.ZMC_EINVAL and "zmc_user_source_1" in str(e.value)
    with pytest.raises(zmc.ZmcError) as e:
        zmc.Udf([HELPER_A, HELPER_B], [1, 13])
    assert e.value.status == zmc.ZMC_EINVAL
