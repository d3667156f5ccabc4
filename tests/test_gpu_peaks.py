"""The library's peak-rate microbenchmarks (deer_measure_peak), the denominators of the
ALU and tensor-pipe rooflines: they run on this GPU, report plausible rates for a GB300
(nominal dense figures: about 80 TFLOP/s FP32 at the top clock, 1.1 PFLOP/s tf32 and 2.25
PFLOP/s bf16 on the tensor cores) and the bf16 tensor rate is about twice the tf32 one."""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    from paper_2603_16850_gb300 import _native as N
    lib = N.load()
    st = torch.cuda.current_stream().cuda_stream
    out = {}
    for name, what in (("fp32", 0), ("fp64", 1), ("tf32", 2), ("bf16", 3)):
        v = C.c_double(0.0)
        assert lib.deer_measure_peak(what, st, C.byref(v)) == N.DEER_OK, name
        out[name] = v.value / 1e12
    assert 30.0 < out["fp32"] < 200.0, out
    assert 0.05 < out["fp64"] < 100.0, out
    assert 300.0 < out["bf16"] < 3000.0, out
    assert 1.5 < out["bf16"] / out["tf32"] < 2.5, out
    v = C.c_double(0.0)
    assert lib.deer_measure_peak(7, st, C.byref(v)) == N.DEER_ERR_INVALID
