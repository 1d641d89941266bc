"""Register and shared-memory budgets of the sm_103a kernels, checked on CPU from
ptxas's resource report (nvcc -Xptxas -v, the flags of the library build).

* No kernel spills registers to local memory.
* The FP64 split-K Gram/projection kernel fits 7 CTAs per SM and the FP32 one 16:
  their splits are sized to one wave of 152 x 7 (152 x 16) CTAs.
* The fused FP32 update + Gram kernel fits 4 CTAs of 256 threads per SM for
  blocks of up to 64 columns and 2 for up to 128, as its slab plan assumes.
* The tensor-core product kernel's 320 threads fit its registers in one SM.
* The cluster Cholesky fits one CTA (256 threads, 133 KB matrix copy) on an SM.
"""

import concurrent.futures as cf
import re
import subprocess

import pytest

from paper_2403_06218_gb300 import build as B

REGS_PER_SM = 65536
SMEM_PER_SM = 228 * 1024       # bytes; 1 KB of it is reserved per resident CTA
MAX_THREADS_PER_SM = 2048
MAX_CTAS_PER_SM = 32


def _ptxas_report(src, tmp):
    cmd = [B._nvcc(), *B.NVCC_FLAGS, "-Xptxas", "-v", "-c", str(src), "-o", str(tmp / (src.stem + ".o"))]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return r.stderr


def _parse(report):
    """{mangled kernel name: {"regs", "smem", "spill_st", "spill_ld"}}"""
    out, cur = {}, None
    for line in report.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = out.setdefault(m.group(1), {"regs": 0, "smem": 0, "spill_st": 0, "spill_ld": 0})
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            cur["spill_st"], cur["spill_ld"] = int(m.group(1)), int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            cur["regs"] = int(m.group(1))
            s = re.search(r"(\d+) bytes smem", line)
            cur["smem"] = int(s.group(1)) if s else 0
    return out


@pytest.fixture(scope="module")
def kernels(tmp_path_factory):
    try:
        B._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    tmp = tmp_path_factory.mktemp("ptxas")
    srcs = B._sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        reports = list(ex.map(lambda s: _ptxas_report(s, tmp), srcs))
    out = {}
    for rep in reports:
        out.update(_parse(rep))
    assert out, "ptxas reported no kernels"
    return out


def _resident_ctas(regs, threads, smem):
    warps = (threads + 31) // 32
    regs_per_warp = (regs * 32 + 255) // 256 * 256          # allocation unit: 256 registers a warp
    by_regs = REGS_PER_SM // (warps * regs_per_warp)
    by_smem = SMEM_PER_SM // (smem + 1024)
    by_threads = MAX_THREADS_PER_SM // threads
    return min(by_regs, by_smem, by_threads, MAX_CTAS_PER_SM)


def _one(kernels, pattern):
    hits = [v for k, v in kernels.items() if re.search(pattern, k)]
    assert len(hits) == 1, (pattern, [k for k in kernels if re.search(pattern, k)])
    return hits[0]


def test_no_kernel_spills(kernels):
    spilling = {k: v for k, v in kernels.items() if v["spill_st"] or v["spill_ld"]}
    assert not spilling, spilling


def test_fp64_split_k_kernel_fits_its_wave(kernels):
    k = _one(kernels, r"gemm_tn_kernelIddE")
    assert _resident_ctas(k["regs"], 128, k["smem"]) >= 7, k


def test_fp32_split_k_kernel_fits_its_wave(kernels):
    # the FP32 split plan targets one wave of 152 x 16 CTAs of 64 threads
    for name in (r"gemm_tn_f32_kernelIdE", r"gemm_tn_f32_kernelIfE"):
        k = _one(kernels, name)
        assert _resident_ctas(k["regs"], 64, k["smem"]) >= 16, k


def test_fused_update_gram_kernel_fits_its_wave(kernels):
    # its slab plan targets one wave of 152 x 4 CTAs of 256 threads for b <= 64 and
    # 152 x 2 for b <= 128
    for name, ctas in ((r"update_gram_f32_kernelILi1E", 4), (r"update_gram_f32_kernelILi2E", 2)):
        k = _one(kernels, name)
        assert _resident_ctas(k["regs"], 256, k["smem"]) >= ctas, k


def test_cluster_cholesky_fits_one_cta_per_sm(kernels):
    # 256 threads and the b x (b + 1) + b doubles of its matrix copy at b = 128 (133 KB
    # of dynamic shared memory): one CTA on each of the cluster's 8 SMs
    k = _one(kernels, r"chol_inv_cluster_kernel")
    dyn = 8 * (128 * 129 + 128)
    assert k["regs"] * 256 <= REGS_PER_SM, k
    assert k["smem"] + dyn + 1024 <= SMEM_PER_SM, k


def test_tensor_core_kernel_fits_one_sm(kernels):
    k = _one(kernels, r"tc_gemm_kernel")
    assert k["regs"] * 320 <= REGS_PER_SM, k


def test_resident_cta_arithmetic():
    # 72 registers x 128 threads: 4 warps x 2304 registers -> 7 CTAs; 16 KB of shared memory allows 13
    assert _resident_ctas(72, 128, 16384) == 7
    # 72 registers x 64 threads: 2 warps x 2304 -> 14 CTAs; 64 registers would allow 16
    assert _resident_ctas(72, 64, 8192) == 14 and _resident_ctas(64, 64, 8192) == 16
