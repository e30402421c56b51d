"""Measurement support: the FP64 fma throughput probe used by bench.py's
FP64-path roofline returns a finite positive rate within the range a
Blackwell-class GPU can have (it is a timing, so only its plausibility is
checked)."""
import math

import pytest

from paper_2101_02286_gb300 import abi

pytestmark = pytest.mark.gpu


def test_fp64_probe_plausible(cuda):
    v = abi.cbs_probe_fp64_peak()
    assert math.isfinite(v) and 0.05 < v < 100.0, v
