"""The L2 read microbenchmark behind the traces' second roofline (needs a B300): a buffer
that fits in L2 reads faster than DRAM can deliver, and the figure is repeatable."""
import pytest
import torch

import paper_2007_14394_b300 as S

pytestmark = pytest.mark.gpu


def test_l2_read_bandwidth_exceeds_dram_and_repeats(cuda_device):
    buf = torch.zeros((32 << 20) // 4, dtype=torch.float32, device="cuda")
    g = [S.l2_read_bandwidth(buf, reps=50) for _ in range(3)]
    print("L2 read GB/s", g)
    assert min(g) > 8000.0  # above the 6.5 TB/s HBM copy rate measured on these parts
    assert max(g) < 1.3 * min(g)
    big = torch.zeros((1 << 30) // 4, dtype=torch.float32, device="cuda")  # 1 GiB: from DRAM
    d = S.l2_read_bandwidth(big, reps=2)
    print("1 GiB read GB/s", d)
    assert d < min(g)
