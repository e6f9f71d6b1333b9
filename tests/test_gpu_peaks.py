"""The pipe microbenchmarks (wos_measure_pipes): every rate measured and
positive, the FP32 FMA and logic pipes far above the SFU and FP64 pipes, and
per SM per clock within a factor of two of the unit counts at the maximum
clock (FFMA 128, LOP3 64 or 128, MUFU 16, DFMA 2 lanes; 128 lanes issued)."""
import pytest
import torch

from gpu_util import ctx
from paper_2409_03686_gb300 import wos

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    p = wos.wos_measure_pipes(ctx())
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per = {k: v / (sms * 2.07e9) for k, v in p.items()}
    assert all(v > 0 for v in p.values()), p
    assert min(per["ffma"], per["lop3"]) > per["mufu"] > per["dfma"], per
    for k, lo, hi in (("ffma", 64, 256), ("lop3", 32, 256), ("mufu", 8, 32), ("dfma", 1, 4),
                      ("issue", 64, 256)):
        assert lo <= per[k] <= hi, (k, per[k])
