"""bench.py's roofline arithmetic (CPU only): the assembly's algorithmic bytes
equal a launch-by-launch count of what each launch of one ChFSI iteration moves
(Eq. chebFilter's degree steps, then the application of H~ in Rayleigh-Ritz),
and the cell kernel's algorithmic flops are N_c 2 n_e^2 per vector and
application (Sec. 3.3.1)."""
import numpy as np
import pytest

import bench
from paper_1903_10959_gb300 import workloads as W


def _launch_by_launch(s, n, block, M, steps, nonlocal_in_assembly):
    """Bytes of every assembly launch of `steps` iterations, column block by block."""
    ncells, ne, sx = s.ncell ** 3, (s.p + 1) ** 3, 4
    total = 0
    for _ in range(steps):
        for b0 in range(0, n, block):
            nb = min(block, n - b0)
            # degree steps k = 1 .. m: R read, Y_out written, Y_in read (shift), Y_prev from k = 2
            for k in range(1, s.degree + 1):
                total += (ncells * ne + M + M + (M if k >= 2 else 0)) * nb * sx
                total += (M + 1 + ncells * ne) * 4
                total += M * nb * sx if nonlocal_in_assembly else 0
            # Rayleigh-Ritz: R read, Y_out written
            total += (ncells * ne + M) * nb * sx + (M + 1 + ncells * ne) * 4
            total += M * nb * sx if nonlocal_in_assembly else 0
    return total


@pytest.mark.parametrize("block", [1100, 200])
@pytest.mark.parametrize("gather,nl", [("rings", False), ("rings", True), ("registers", True)])
def test_assembly_bytes_match_a_launch_by_launch_count(block, gather, nl):
    s = W.fcc_periodic()
    if nl:
        s.nl_centres = s.centres[:4].copy()
    n, M, steps = 1100, (s.ncell * s.p) ** 3, 3
    nblocks = -(-n // block)
    steps_blocks = steps * (s.degree + 1)
    launches = steps_blocks * nblocks
    peaks = {"hbm_gbs": 6700.0, "bf16_tflops_sustained": 1744.4, "source": "test"}
    roof, asm, step = bench.rooflines("bf16x3", s, n, M, peaks, steps_blocks * n, steps_blocks, nblocks,
                                      5.0 * launches, launches, 3.0 * launches, launches, gather=gather)
    in_asm = nl and gather not in ("rings", "rings4")
    want = _launch_by_launch(s, n, block, M, steps, in_asm)
    assert asm["bytes_per_launch"] * launches == pytest.approx(want, rel=1e-12)
    # cell kernel: N_c 2 n_e^2 flops per vector and application
    ne = (s.p + 1) ** 3
    assert roof["flops_per_launch"] * launches == pytest.approx(s.ncell ** 3 * 2 * ne * ne * n * steps_blocks,
                                                                 rel=1e-12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / peaks["bf16_tflops_sustained"])
