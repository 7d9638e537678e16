"""Register and local-memory budgets of the step kernels, from ptxas's resource report.

The 3D step kernel marches a 9-deep register queue per cell; any per-thread array that the
compiler cannot keep in registers (a spill, or an array indexed at run time) puts a local-
memory round trip on every plane, which cost 2 % of the 400^3 throughput when the point-
source sum was added through an index.  Every variant must have no stack frame, and the FP32
variants must fit the three blocks of 160 threads per SM that the shared-memory ring allows.
Compiles one translation unit with nvcc (no GPU needed)."""
import os
import re
import shutil
import subprocess

import pytest

from paper_2211_06300_gb300 import build

pytestmark = pytest.mark.skipif(
    not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")),
    reason="nvcc not available")


def _ptxas_report(src, tmp_path):
    cmd = [build.nvcc()] + build.ARCH + build.FLAGS + [
        "-Xptxas", "-v", "-c", os.path.join(build.CSRC, src), "-o", str(tmp_path / "k.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, name, rows = r.stdout + r.stderr, None, {}
    for line in out.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and name:
            rows.setdefault(name, {})["stack"] = int(m.group(1))
            rows[name]["spill"] = int(m.group(2)) + int(m.group(3))
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            rows.setdefault(name, {})["regs"] = int(m.group(1))
    return rows


def test_3d_step_variants_keep_their_state_in_registers(tmp_path):
    rows = _ptxas_report("fd3d.cu", tmp_path)
    step = {k: v for k, v in rows.items() if "fd3_step_kernel" in k}
    assert len(step) >= 30, sorted(rows)          # 15 flag sets x {FP32, FP64}
    for k, v in step.items():
        assert v["stack"] == 0 and v["spill"] == 0, (k, v)
        if "fd3_step_kernelIf" in k:
            # 3 blocks x 160 threads within the SM's 65,536 registers
            assert v["regs"] * 160 * 3 <= 65536, (k, v)


def test_2d_cg_product_halves_stay_within_their_register_budget(tmp_path):
    """The two halves of the 2D CG product (`fd2_step[CGP|SMP]`, `fd2_step[PT|AP]`) run at
    4 blocks of 256 threads per SM, i.e. 64 registers; the forward half fits without spills
    and the adjoint half spills at most 16 bytes."""
    rows = _ptxas_report("fd2d.cu", tmp_path)
    f32 = {k: v for k, v in rows.items() if "fd2_step_kernelIf" in k}
    assert f32, sorted(rows)
    for k, v in f32.items():
        assert v["regs"] <= 64, (k, v)
    cgp = [v for k, v in f32.items() if "fd2_step_kernelIfLj10E" in k]   # CGP | SMP
    ap = [v for k, v in f32.items() if "fd2_step_kernelIfLj36E" in k]    # PT | AP
    assert len(cgp) == 1 and len(ap) == 1
    assert cgp[0]["stack"] == 0 and cgp[0]["spill"] == 0, cgp
    assert ap[0]["spill"] <= 32, ap        # 16 bytes stored + 16 loaded
