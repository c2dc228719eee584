"""The integrator converts between double and float with integer operations
on the IEEE-754 fields (the conversion instructions run on the FP64 pipe).
Those conversions must give exactly what the instructions give (round to
nearest, ties to even): checked on the device over hashed inputs, a
quarter of them on rounding ties and a quarter with exponents around the
float range, through dem_check_conversions."""
import pytest

from tests.gpu_common import load_dem

pytestmark = pytest.mark.gpu


def test_conversions_match_instructions():
    dem = load_dem()
    for seed in (1, 1607_02427):
        assert dem.dem_check_conversions(1 << 28, seed) == (0, 0)


def test_conversions_rejects_null():
    import ctypes as C
    dem = load_dem()
    assert dem.load().dem_check_conversions(C.c_ulonglong(16), C.c_ulonglong(0), None) == dem.DEM_ERR_ARG
