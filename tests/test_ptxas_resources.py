"""Register and spill budgets of the hot kernels at the 256-, 384- and 144-point lengths (the 128^3 bench
grid, the serving mix's 192^3 grids, the bead at lambda/16), from ptxas's resource report (no GPU).  The
occupancy each pass is designed for depends on these numbers: at L = 256 the TMA z pass runs two 288-thread
CTAs per SM (at most 113 registers a thread), the FFT passes several CTAs per SM."""
import os
import re
import shutil
import subprocess

import pytest

NVCC = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else
                                  shutil.which("nvcc"))

# transform length -> kernel (demangled-name prefix) -> (max registers, max spill-store bytes)
BUDGET = {
    256: {  # the 128^3 bench grid
        "k_zw<256, false, false>": (96, 0),     # z pass one CTA per tile, two 288-thread CTAs per SM
        "k_zw<256, false, true>": (96, 0),      # the same, static persistent
        "k_zwd<256>": (96, 0),                  # the dynamically scheduled z pass
        "k_strided<256, -1, 16>": (48, 0),      # FY, five resident 256-thread CTAs
        "k_strided<256, 1, 16>": (48, 0),       # IY
        "k_ix<256>": (48, 0),                   # IX, five resident 256-thread CTAs
        "k_fxb<256>": (96, 0),                  # FX bulk-staged (persistent, one CTA per SM)
        "k_fx<256>": (40, 16),                  # FX: six resident CTAs at 40 registers, a few bytes of spill
    },
    384: {  # 192^3 grids of the serving mix
        "k_zw<384, false, false>": (168, 0),    # one CTA per SM; Green values of both sub-transforms in registers
        "k_zwd<384>": (168, 0),
        "k_strided3<384, -1, 16>": (56, 8),     # FY: three resident 384-thread CTAs
        "k_strided3<384, 1, 16>": (56, 8),      # IY
        "k_ix<384>": (56, 0),                   # IX, six resident 192-thread CTAs
        "k_fx<384>": (56, 0),
    },
    144: {  # the Fig. 3 bead at lambda/16
        "k_zg<144, false>": (80, 0),            # column-group z pass
        "k_zg<144, true>": (80, 4),             # its persistent form
        "k_strided<144, -1, 16>": (40, 0),
        "k_strided<144, 1, 16>": (40, 0),
        "k_ix<144>": (56, 0),                   # IX, six resident 192-thread CTAs
        "k_fx<144>": (56, 0),
    },
}
CASES = [(L, k) for L in sorted(BUDGET) for k in sorted(BUDGET[L])]


def _demangle(names):
    r = subprocess.run(["c++filt"], input="\n".join(names), capture_output=True, text=True)
    return r.stdout.splitlines() if r.returncode == 0 else names


@pytest.fixture(scope="module")
def resources(tmp_path_factory, repo_root):
    if not NVCC or shutil.which("c++filt") is None:
        pytest.skip("nvcc or c++filt not available")
    csrc = os.path.join(repo_root, "paper_1910_13844_gb300", "csrc")
    tmp = tmp_path_factory.mktemp("ptxas")
    cache = {}

    def report(L):
        if L in cache:
            return cache[L]
        r = subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
                            "--expt-relaxed-constexpr", "-O3", "-I", os.path.join(repo_root, "include"), "-I", csrc,
                            "-Xptxas", "-v", "-c", os.path.join(csrc, f"passes_L{L}.cu"), "-o", str(tmp / f"p{L}.o")],
                           capture_output=True, text=True, timeout=600)
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
        cache[L] = {d: entries[n] for n, d in zip(names, _demangle(names))}
        return cache[L]
    return report


@pytest.mark.parametrize("length,kernel", CASES)
def test_kernel_stays_within_its_register_and_spill_budget(resources, length, kernel):
    found = resources(length)
    hits = [v for k, v in found.items() if k.startswith(f"void lsgpu::{kernel}(")]
    assert len(hits) == 1, sorted(found)
    regs, spill = BUDGET[length][kernel]
    assert hits[0]["regs"] <= regs, hits[0]
    assert hits[0]["spill"] <= spill, hits[0]
