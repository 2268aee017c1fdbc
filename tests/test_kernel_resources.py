"""Register and spill budgets of the hot kernels, from ptxas's resource report
(`nvcc -Xptxas -v` for sm_103a, no GPU needed): no kernel on a default path
spills to local memory, and each fits the occupancy its launch is designed
for (the FP32 analysis kernel: two 128-thread CTAs per SM, so at most 256
registers; the spin-2 kernel: three 128-thread CTAs, as its launch bounds
state; the mma.sync weight-column kernel: one 256-thread CTA)."""
import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2312_12285_gb300", "csrc")

# file -> [(substring of the mangled kernel name, register ceiling)]
BUDGETS = {
    "analysis.cu": [("15analysis_kernelINS_9TraitsF32ELi16ELi4ELb1EE", 256),   # default FP32 (packed f32x2)
                    ("15analysis_kernelINS_9TraitsF64ELi4ELi4ELb0EE", 255)],   # FP64
    "mixed.cu": [("21analysis_mixed_kernelILi8ELb0EE", 255), ("21analysis_mixed_kernelILi4ELb0EE", 255),
                 ("21analysis_mixed_kernelILi8ELb1EE", 255)],                  # column and table modes
    "mixed_tc.cu": [("18analysis_tc_kernelILi8ELi32EE", 255), ("18analysis_tc_kernelILi4ELi64EE", 255),
                    ("18analysis_tc_kernelILi2ELi128EE", 255)],
    "adjoint.cu": [("21adjoint_sorted_kernel", 255)],
    "spin2.cu": [("18s2_analysis_kernel", 170)],
    "interp.cu": [("13ip_bin_kernel", 255)],
}


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def _resources(nvcc, src, out):
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler",
                        "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v", "-c",
                        os.path.join(CSRC, src), "-o", out], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res, cur, spill = {}, None, None
    for line in r.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            cur, spill = m.group(1), None
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur:
            spill = (int(m.group(1)), int(m.group(2)))
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            res[cur] = (int(m.group(1)), spill)
            cur = None
    return res


def test_hot_kernels_fit_their_register_budgets(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    with ThreadPoolExecutor(len(BUDGETS)) as ex:
        futs = {src: ex.submit(_resources, nvcc, src, str(tmp_path / (src + ".o"))) for src in BUDGETS}
        reports = {src: f.result() for src, f in futs.items()}
    for src, wanted in BUDGETS.items():
        for key, ceiling in wanted:
            hits = [(name, v) for name, v in reports[src].items() if key in name]
            assert len(hits) == 1, (src, key, sorted(reports[src]))
            name, (regs, spill) = hits[0]
            assert spill == (0, 0), (name, spill)
            assert regs <= ceiling, (name, regs, ceiling)
