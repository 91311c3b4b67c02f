"""Resource limits the cycle kernel's speed depends on, read from ptxas's report of the build (no GPU
needed).  Two CTAs of 256 threads per SM, with the dynamic shared memory of the residual stages
(93,760 bytes) and the static tables, must fit the 196 KB shared-memory carveout that leaves L1 its
60 KB (a few hundred bytes more moved the carveout to 228 KB and cost 10 % of the solve), within 128
registers a thread; the mixed-form 3-D kernel (the benchmark's) must not spill."""
import os
import re

import pytest

from paper_1703_07206_gb300 import build

DYNAMIC_SMEM = 93760        # bytes per CTA: kOuterStages stages of the FP64 residual's halo tiles
CARVEOUT = 196 * 1024       # shared-memory carveout that leaves L1 60 KB of the SM's 256 KB
RESERVED_PER_CTA = 1024     # shared memory the hardware reserves per CTA


def report(tag):
    path = os.path.join(build.BUILD, f"ptxas_{tag}.log")
    if not os.path.exists(path):
        build.build(force=True)
    with open(path) as fh:
        return fh.read()


def cycle_kernels(text):
    """{(T, DIM): (registers, static smem, spill stores, spill loads)} of the cycle kernels."""
    out = {}
    blocks = re.split(r"ptxas info\s*: Compiling entry function '", text)
    for blk in blocks[1:]:
        name = blk.split("'", 1)[0]
        m = re.search(r"cycle_kernelI([fd])Li([23])E", name)
        if not m:
            continue
        regs = int(re.search(r"Used (\d+) registers", blk).group(1))
        smem = re.search(r"(\d+) bytes smem", blk)
        spills = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", blk)
        out[(m.group(1), int(m.group(2)))] = (regs, int(smem.group(1)) if smem else 0,
                                             int(spills.group(1)), int(spills.group(2)))
    return out


@pytest.mark.parametrize("tag", ["k64", "k32"])
def test_two_ctas_per_sm_fit_the_carveout(tag):
    k = cycle_kernels(report(tag))
    assert set(k) == {("f", 2), ("f", 3), ("d", 2), ("d", 3)}, k
    for key, (regs, static, _, _) in k.items():
        assert regs <= 128, (key, regs)
        assert 2 * (DYNAMIC_SMEM + static + RESERVED_PER_CTA) <= CARVEOUT, (key, static)


def test_mixed_form_kernel_does_not_spill():
    regs, static, stores, loads = cycle_kernels(report("k64"))[("f", 3)]
    assert stores == 0 and loads == 0, (stores, loads)
