"""The pipe microbenchmarks (wos_measure_pipes): every rate measured and
positive, in the order the unit counts give (FP32 FMA above the half-rate
logic pipe, both far above the SFU and FP64 pipes), and per SM per clock
within a factor of two of those unit counts at the maximum clock (FFMA 128,
LOP3 64, MUFU 16, DFMA 2 lanes; 128 lanes issued)."""
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
    assert per["ffma"] > per["lop3"] > per["mufu"] > per["dfma"], per
    for k, nominal in (("ffma", 128), ("lop3", 64), ("mufu", 16), ("dfma", 2), ("issue", 128)):
        assert nominal / 2 <= per[k] <= nominal * 2, (k, per[k])
