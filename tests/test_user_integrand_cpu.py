"""User integrands compiled with NVRTC: registration and validation need no GPU."""
import numpy as np
import pytest

import user_sources as us


@pytest.fixture(scope="module")
def z():
    from paper_1910_01965_gb300 import build, zmc
    build.build()
    zmc.load()
    try:
        zmc.zmc_integrand_register("probe", us.SUMX_PRODY, 1, 2)
    except zmc.ZmcError as e:
        if e.status == zmc.ZMC_ENOTFOUND:
            pytest.skip("NVRTC not available: %s" % e)
        raise
    return zmc


def test_register_and_describe(z):
    gid = z.zmc_integrand_register("cosprod_user", us.COSPROD, 1, 8)
    assert gid >= z.ZMC_G_USER_BASE
    assert z.zmc_integrand_info_get(gid).name == b"cosprod_user"
    assert z.zmc_integrand_info_get(gid).m_rule == 0


def test_compile_errors_come_back_with_the_log(z):
    with pytest.raises(z.ZmcError) as e:
        z.zmc_integrand_register("broken", us.BROKEN)
    assert e.value.status == z.ZMC_EINVAL and "expected an expression" in str(e.value)


def test_validation_of_user_scans(z):
    gid = z.zmc_integrand_register("sumx_prody", us.SUMX_PRODY, 2, 3)  # FP32 only
    ok, k1 = z.make_desc(gid, 2, [0, 0], [1, 2], [3, 2], np.arange(5.0), 64, 2, 0)
    assert z.zmc_validate(ok) == 0
    bad_n, k2 = z.make_desc(gid, 4, [0] * 4, [1] * 4, [3], np.arange(3.0), 64, 2, 0)
    assert z.zmc_validate(bad_n) == z.ZMC_EINVAL
    no64, k3 = z.make_desc(gid, 2, [0, 0], [1, 2], [3], np.arange(3.0), 64, 2, 0,
                           precision=z.ZMC_FP64)
    assert z.zmc_validate(no64) == z.ZMC_EINVAL and "zmc_user_g64" in z.zmc_last_error()
    unknown, k4 = z.make_desc(z.ZMC_G_USER_BASE + 63, 2, [0, 0], [1, 1], [3], np.arange(3.0),
                              64, 2, 0)
    assert z.zmc_validate(unknown) == z.ZMC_ENOTFOUND
