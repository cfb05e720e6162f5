"""Arithmetic peaks of this GPU, measured: double and single precision FMA throughput of long
independent FMA chains over a full grid (tests/cuda/fp_peak.cu).  The FP64 form is bound by the
FP64 pipe; this measured double rate is the denominator its roofline fraction can be read against
(the bench reports the rate derived from unit counts and clocks, 152 SMs x 2 FMA x 2 flop x
2.07 GHz).  The measured figures are printed on a line starting with "MEASURED"."""
import ctypes as C
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fp64_and_fp32_fma_throughput(tmp_path):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    out = str(tmp_path / "libpeak.so")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "cuda", "fp_peak.cu")], check=True, capture_output=True)
    lib = C.CDLL(out)
    lib.fp_peak.restype = C.c_double
    lib.fp_peak.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp64 = max(lib.fp_peak(0, sms * 8, 256, 200) for _ in range(3))
    fp32 = max(lib.fp_peak(1, sms * 8, 256, 2000) for _ in range(3))
    print("MEASURED " + json.dumps({"fp64_tflops": fp64 / 1e12, "fp32_tflops": fp32 / 1e12, "sms": sms,
                                    "device": torch.cuda.get_device_name(0)}), flush=True)
    assert fp64 > 0 and fp32 > 0
    assert fp32 > 10 * fp64  # a part with reduced FP64 throughput, as the FP64 form's design assumes
