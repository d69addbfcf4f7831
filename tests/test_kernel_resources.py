"""Resource budgets of the hot kernels, read from ptxas's resource summary
(-Xptxas -v) on the CPU: the register counts that set how many CTAs fit per SM
and the absence of spills, which the measured throughputs depend on. A change
that breaks one of them shows up here before it reaches a GPU."""
import os
import re
import subprocess
import tempfile

import pytest

from paper_2609_02876_gb300 import build as B


def resources(src, extra=()):
    """{mangled kernel name: (registers, spill store bytes)} for one translation unit."""
    with tempfile.TemporaryDirectory() as tmp:
        cmd = [B.nvcc()] + B.ARCH + B.FLAGS + list(extra) + ["-Xptxas", "-v", "-c", os.path.join(B.CSRC, src),
                                                             "-o", os.path.join(tmp, "k.o")]
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    out, cur, spill = {}, None, 0
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            cur, spill = m.group(1), 0
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and cur:
            spill = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            out[cur] = (int(m.group(1)), spill)
            cur = None
    return out


def find(res, *parts):
    hits = [v for k, v in res.items() if all(p in k for p in parts)]
    assert len(hits) == 1, (parts, [k for k in res if all(p in k for p in parts)])
    return hits[0]


@pytest.fixture(scope="module")
def tsit5():
    return resources("gs_tsit5.cu")


def test_lorenz_fp64_stored_stage_kernels_fit_four_ctas_without_spills(tsit5):
    # 128 threads per CTA: at most 128 registers for 4 CTAs (16 warps) per SM
    regs, spill = find(tsit5, "record_kernel", "Tsit5Method", "Lorenz", "EdLb1ELb1ELb0E")
    assert regs <= 128 and spill == 0
    # the stored-stage reverse sweep is capped at 5 CTAs per SM (96 registers; a small spill)
    regs, spill = find(tsit5, "reverse_k1_kernel_mb", "Tsit5Method", "Lorenz", "EdLb0ELb1ELi5E")
    assert regs <= 96 and spill <= 512
    # the same record with FP64 step control (the library pow and division)
    regs, spill = find(tsit5, "record_kernel", "Tsit5Method", "Lorenz", "EdLb1ELb1ELb1E")
    assert regs <= 128 and spill == 0


def test_fp32_mixed_kernels_stay_small(tsit5):
    regs, spill = find(tsit5, "record_kernel", "Tsit5Method", "Lorenz", "EfLb0ELb0ELb0E")
    assert regs <= 80 and spill == 0
    # the FP32-mixed reverse sweep is capped at 8 CTAs per SM (64 registers)
    regs, spill = find(tsit5, "reverse_k1_kernel_mb", "Tsit5Method", "Lorenz", "EfLb0ELb0ELi8E")
    assert regs <= 64 and spill <= 64


def test_ude_reverse_fits_three_ctas(tsit5):
    # 3 CTAs of 128 threads per SM need at most 170 registers
    regs, _ = find(tsit5, "reverse_k1_kernel", "Tsit5Method", "LvUdeWarp", "EfLb0ELb0E")
    assert regs <= 170


def test_verner7_stored_stage_kernels():
    res = resources("gs_vern7.cu")
    regs, spill = find(res, "record_kernel", "Verner7Method", "Lorenz", "EdLb1ELb1E")
    assert regs <= 128 and spill == 0  # 4 CTAs per SM
    regs, spill = find(res, "reverse_k1_kernel", "Verner7Method", "Lorenz", "EdLb0ELb1E")
    assert regs <= 170 and spill == 0  # 3 CTAs per SM


def test_tcgen05_ude_variant_builds():
    """The CTA-collective UDE network (hidden layer on tcgen05, TMEM accumulator)
    is the compile-time alternative of the reverse sweep (GS_UDE_CTA=1): it must
    keep compiling for sm_103a, within 3 CTAs' registers and without spills."""
    res = resources("gs_tsit5.cu", ["-DGS_UDE_CTA=1"])
    regs, spill = find(res, "reverse_k1_kernel", "Tsit5Method", "LvUdeCta", "EfLb0ELb0E")
    assert regs <= 168 and spill == 0
