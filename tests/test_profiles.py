"""The committed ncu summaries stay consistent with the tree.

Every summary under profiles/ gives the command that produced it; every ncu
command there leaves the GPU clocks alone (--clock-control none) and runs
committed files only; a summary that records a kernel's source hash matches
the current source of that kernel (bench.py takes the headline kernel's DRAM
traffic from such a summary only while the hashes agree)."""
import hashlib
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")
CSRC = os.path.join(ROOT, "paper_1712_08740_gb300", "csrc")


def summaries():
    return sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))


def kernel_hash(src, kernel, bounds):
    code = open(os.path.join(CSRC, src)).read()
    m = re.search(r"__global__ void __launch_bounds__\(" + re.escape(bounds) + r"\)\nk_" + kernel + r"\(.*?\n}\n",
                  code, re.S)
    assert m, (src, kernel)
    return hashlib.sha256(m.group(0).encode()).hexdigest()[:16]


@pytest.mark.parametrize("name", summaries())
def test_summary_states_its_command(name):
    lines = open(os.path.join(PROFILES, name)).read().split("\n")
    cmds = []
    for i, ln in enumerate(lines):          # fenced or indented command lines, with continuations
        if ln.strip().startswith("ncu "):
            parts = [ln.strip()]
            while parts[-1].endswith("\\") and i + 1 < len(lines):
                i += 1
                parts[-1] = parts[-1][:-1]
                parts.append(lines[i].strip())
            cmds.append(" ".join(parts))
    assert cmds, f"{name}: no ncu command"
    for joined in cmds:
        assert "--clock-control none" in joined, name
        assert "_work" not in joined and "/root/" not in joined, name
        # the profiled program is a committed file of the repository
        prog = re.search(r"python (\S+\.py)", joined)
        assert prog and os.path.exists(os.path.join(ROOT, prog.group(1))), (name, joined)


def test_recorded_kernel_hashes_match_the_source():
    checks = [("k_multidot_h_2d_smooth_401x201.md", [("krylov.cu", "multidot_h", "kThreads")]),
              ("k_multidot_sb_k_multiaxpy_sb_401x201_64rhs.md",
               [("krylov_ds.cu", "multidot_sb", "kPipeThreads, kDotBlocksPerSM"),
                ("krylov_ds.cu", "multiaxpy_sb", "kPipeThreads, kAxpyBlocksPerSM")])]
    for name, kernels in checks:
        text = open(os.path.join(PROFILES, name)).read()
        recorded = re.findall(r"[0-9a-f]{16}", text.split("kernel_source_sha256_16", 1)[1].split("\n", 1)[0])
        assert recorded, name
        for k, (src, kernel, bounds) in enumerate(kernels):
            assert kernel_hash(src, kernel, bounds) == recorded[k], (name, kernel)
