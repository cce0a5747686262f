"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function that the headers under include/ declare (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(mlmc(?:3d|p|c)?_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mlmc_create", "mlmc_destroy", "mlmc_sample_level", "mlmc_solve_batch",
                     "mlmc_estimate", "mlmc_last_error", "mlmc3d_create", "mlmc3d_sample_level",
                     "mlmc3d_solve_batch", "mlmcp_create", "mlmcp_sample_level", "mlmcp_solve_batch",
                     "mlmcc_create", "mlmcc_sample_level", "mlmcc_sample_levels", "mlmcc_solve_batch"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1907_10271_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1907_10271_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        binding.lib()


def test_config_marshalling():
    from paper_1907_10271_gb300 import binding
    from workloads import STRIP_MIXED_5LEVEL
    c = binding.config_from_workload(STRIP_MIXED_5LEVEL)
    assert (c.nx0, c.ny0, c.levels, c.kl_terms) == (64, 16, 5, 100)
    assert c.precision == binding.MLMC_PREC_MIXED
    assert abs(c.kl_std - 2.0 * 3.141592653589793 / 180.0) < 1e-15


def test_config3_marshalling():
    from paper_1907_10271_gb300 import binding
    from workloads import HEX8_MIXED_4LEVEL
    c = binding.config3_from_workload(HEX8_MIXED_4LEVEL)
    assert (c.nx0, c.ny0, c.nz0, c.levels, c.kl_terms) == (32, 8, 4, 4, 200)
    assert (c.G23, c.nu23, c.lz) == (3.5e9, 0.45, 0.125)
    assert abs(c.kl_std - 3.0 * 3.141592653589793 / 180.0) < 1e-15


@pytest.mark.parametrize("override,msg", [(dict(ly=0.3), "cubes"), (dict(levels=0), "levels"),
                                          (dict(kl_terms=0), "kl_terms"), (dict(rtol=0.0), "rtol"),
                                          (dict(nx0=4, ny0=1, nz0=1, lx=1.0, ly=0.25, lz=0.25), "mesh too small")])
def test_create3_rejects_invalid_configs_without_a_gpu(override, msg):
    # validation runs before any CUDA call, so it answers on a machine without a GPU
    from paper_1907_10271_gb300 import binding
    from workloads import HEX8_MIXED_4LEVEL
    with pytest.raises(binding.MLMCError, match=msg):
        binding.mlmc3d_create(binding.config3_from_workload(HEX8_MIXED_4LEVEL, **override), stream=0)


def test_configp_marshalling():
    from paper_1907_10271_gb300 import binding
    from workloads import PANEL_RM_4LEVEL
    c = binding.configp_from_workload(PANEL_RM_4LEVEL)
    assert (c.nx0, c.ny0, c.levels, c.n_plies, c.hard_support) == (24, 8, 4, 8, 1)
    assert list(c.plies_deg[:8]) == [45.0, -45.0, -45.0, 45.0, -45.0, 45.0, 45.0, -45.0]
    assert (c.t_ply, c.ply_std_deg, c.p_star, c.lx, c.ly) == (0.8, 3.0, 272.47, 636.0, 212.0)
    assert binding.configp_from_workload(PANEL_RM_4LEVEL, bc="soft").hard_support == 0


@pytest.mark.parametrize("override,msg", [(dict(levels=0), "levels"), (dict(t_ply=0.0), "thickness"),
                                          (dict(nx0=25), "coarsest"), (dict(tol=-1.0), "tolerances"),
                                          (dict(G13=0.0), "moduli")])
def test_createp_rejects_invalid_configs_without_a_gpu(override, msg):
    # validation runs before any CUDA call, so it answers on a machine without a GPU
    from paper_1907_10271_gb300 import binding
    from workloads import PANEL_RM_4LEVEL
    with pytest.raises(binding.MLMCError, match=msg):
        binding.mlmcp_create(binding.configp_from_workload(PANEL_RM_4LEVEL, **override), stream=0)
