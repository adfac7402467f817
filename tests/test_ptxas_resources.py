"""Register and spill budget of the 256-point kernels (the 128^3 workload's path), from ptxas's resource
report (no GPU).  The occupancy the passes are designed for depends on these numbers: the TMA z pass runs
two 288-thread CTAs per SM (at most 113 registers a thread), the FFT passes several CTAs per SM."""
import os
import re
import shutil
import subprocess

import pytest

NVCC = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else
                                  shutil.which("nvcc"))

# kernel (demangled-name prefix) -> (max registers, max spill-store bytes)
BUDGET = {
    "k_zw<256, false, false>": (96, 0),     # the z pass one CTA per tile (default at large batches)
    "k_zw<256, false, true>": (96, 0),      # the same, static persistent
    "k_zwd<256>": (96, 0),                  # the dynamically scheduled z pass
    "k_strided<256, -1, 16>": (48, 0),      # FY, five resident 256-thread CTAs
    "k_strided<256, 1, 16>": (48, 0),       # IY
    "k_ix<256>": (48, 0),                   # IX, five resident 256-thread CTAs
    "k_fxb<256>": (96, 0),                  # FX bulk-staged (persistent, one CTA per SM)
    "k_fx<256>": (40, 16),                  # FX: six resident CTAs at 40 registers, a few bytes of spill
}


def _demangle(names):
    r = subprocess.run(["c++filt"], input="\n".join(names), capture_output=True, text=True)
    return r.stdout.splitlines() if r.returncode == 0 else names


@pytest.fixture(scope="module")
def resources(tmp_path_factory, repo_root):
    if not NVCC or shutil.which("c++filt") is None:
        pytest.skip("nvcc or c++filt not available")
    csrc = os.path.join(repo_root, "paper_1910_13844_gb300", "csrc")
    out = tmp_path_factory.mktemp("ptxas") / "p256.o"
    r = subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                        "-O3", "-I", os.path.join(repo_root, "include"), "-I", csrc, "-Xptxas", "-v", "-c",
                        os.path.join(csrc, "passes_L256.cu"), "-o", str(out)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    entries, cur = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
            entries[cur] = {}
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m:
            entries[cur]["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            entries[cur]["regs"] = int(m.group(1))
    names = list(entries)
    return {d: entries[n] for n, d in zip(names, _demangle(names))}


@pytest.mark.parametrize("kernel", sorted(BUDGET))
def test_kernel_stays_within_its_register_and_spill_budget(resources, kernel):
    hits = [v for k, v in resources.items() if k.startswith(f"void lsgpu::{kernel}(")]
    assert len(hits) == 1, sorted(resources)
    regs, spill = BUDGET[kernel]
    assert hits[0]["regs"] <= regs, hits[0]
    assert hits[0]["spill"] <= spill, hits[0]
