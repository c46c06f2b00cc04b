"""Throughput arithmetic shared by the benchmark and the tests.

Bandwidth is algorithmic bytes / seconds with GB = 1e9 bytes, the convention
of the paper's Table 2 (its bandwidth column is n*4 bytes / time)."""


def gbs(nbytes: float, seconds: float) -> float:
    return nbytes / seconds / 1e9


def frac(achieved: float, peak: float) -> float:
    return achieved / peak
