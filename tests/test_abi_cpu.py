"""Host-side checks of the C-ABI library that need no GPU: it loads and exports
every entry point include/ctt_mg.h declares, and the ctypes structs match the
header's layout."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctt_mg.h")
UNET_HEADER = os.path.join(ROOT, "include", "ctt_unet.h")


def declared_functions(header=HEADER, prefix="mg_"):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(%s[a-z_0-9]+)\s*\(" % prefix, text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import mg
    return mg


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "mg_solve" in names and "mg_create" in names and "mg_residual_norms" in names
    raw = C.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
    assert set(names) <= set(lib.EXPORTS) | {"mg_config_default"}


def test_library_exports_every_network_entry_point(lib):
    names = declared_functions(UNET_HEADER, "unet_")
    assert "unet_conv3d_fwd" in names and "unet_conv3d_fwd_workspace" in names
    raw = C.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_split_convolution_workspace_query(lib):
    """Host-side plan of the split-K per-tap convolutions: grids with fewer than 4 x 152 tiles of
    128 voxels split the 27 taps into groups for about four CTAs per SM; the workspace holds one
    FP32 partial per group, voxel and output channel."""
    from paper_2501_13046_gb300 import unet as U
    f = 4

    def groups(tiles):
        want = min(27, -(-608 // tiles))
        tpg = -(-27 // want)
        return -(-27 // tpg)

    assert groups(4) == 27 and groups(32) == 14 and groups(256) == 3
    assert U.conv3d_workspace((8, 8, 8), 64) == 27 * 512 * 64 * f          # 4 tiles: one tap per group
    assert U.conv3d_workspace((16, 16, 16), 64) == 14 * 4096 * 64 * f      # 32 tiles: 2 taps per group
    assert U.conv3d_workspace((32, 32, 32), 32) == 3 * 32768 * 32 * f      # 256 tiles: 9 taps per group
    assert U.conv3d_workspace((64, 32, 38), 16) == 0                        # 608 tiles: unsplit
    assert U.conv3d_workspace((64, 64, 64), 16) == 0
    assert U.conv3d_workspace((8, 8, 3), 16) == 0                           # not a multiple of 128 voxels
    assert U.conv3d_workspace((0, 8, 8), 16) == 0


def test_config_defaults_and_workspace_size(lib):
    cfg = lib.mg_config_default()
    assert cfg.order == 2 and cfg.tol == 1e-10 and cfg.precision == lib.MG_MIXED and cfg.use_graph == 1
    cfg.n[0] = cfg.n[1] = cfg.n[2] = 32
    nbytes = lib.mg_workspace_size(cfg)
    N = 32 ** 3
    # FP64 state (4), sources (5), pass-1 output (5), q / div W (4) plus FP32 levels (13 arrays, 8/7 geometric)
    assert nbytes >= 18 * 8 * N + 13 * 4 * N
    assert nbytes <= 18 * 8 * N + 13 * 4 * N * 8 // 7 + 2 ** 20
    assert cfg.smoother == 0 and cfg.block_threads == 0


def test_nested_workspace_holds_the_half_size_contexts(lib):
    """nested = 1 adds the half-size problem's workspace, recursively, while every size stays
    even and the half size >= nested_min (default 64): 256^3 nests 128^3, which nests 64^3."""
    def ws(n, nested, nmin=0, order=4):
        cfg = lib.mg_config_default()
        cfg.n[0] = cfg.n[1] = cfg.n[2] = n
        cfg.order, cfg.nested, cfg.nested_min = order, nested, nmin
        return lib.mg_workspace_size(cfg)
    assert ws(64, 1) == ws(64, 0)
    assert ws(128, 1) == ws(128, 0) + ws(64, 0)
    assert ws(256, 1) == ws(256, 0) + ws(128, 1)
    assert ws(40, 1, 24) == ws(40, 0)      # half size 20 < 24: not eligible
    assert ws(48, 1, 24) == ws(48, 0) + ws(24, 0)
    assert ws(128, 1, 24) == ws(128, 0) + ws(64, 1, 24)
    assert ws(64, 1, 24) == ws(64, 0) + ws(32, 1, 24) and ws(32, 1, 24) == ws(32, 0)
    assert ws(128, 1, 24) - ws(128, 0) < ws(128, 0) // 6   # about 1/8 + 1/64, plus the coarse inverses


def test_bowen_york_workspace_and_validation(lib):
    """A puncture with a momentum or spin adds its curvature table (6 FP64 fields) to the
    workspace; a non-finite momentum is rejected on the host."""
    def cfg_for(P=(0.0, 0.0, 0.0), S=(0.0, 0.0, 0.0)):
        cfg = lib.mg_config_default()
        cfg.n[0] = cfg.n[1] = cfg.n[2] = 32
        cfg.bc, cfg.k_mode, cfg.npunct, cfg.punct_m[0] = lib.MG_BC_ROBIN, lib.MG_K_FIXED, 1, 1.0
        for a in range(3):
            cfg.punct_P[0][a], cfg.punct_S[0][a] = P[a], S[a]
        return cfg
    bare = lib.mg_workspace_size(cfg_for())
    assert lib.mg_workspace_size(cfg_for(P=(0.1, 0.0, 0.0))) == bare + 6 * 32 ** 3 * 8
    assert lib.mg_workspace_size(cfg_for(S=(0.0, 0.0, 0.2))) == bare + 6 * 32 ** 3 * 8
    with pytest.raises(lib.MGError) as e:
        lib.mg_workspace_size(cfg_for(P=(float("nan"), 0.0, 0.0)))
    assert e.value.status == lib.MG_ERR_INVALID_ARG


def test_symmetry_plane_validation(lib):
    """reflect needs a Robin box whose marked lower faces are x_a = 0; it adds no workspace."""
    def cfg_for(bc, reflect, lo=0.0):
        cfg = lib.mg_config_default()
        cfg.n[0] = cfg.n[1] = cfg.n[2] = 32
        cfg.bc, cfg.k_mode, cfg.reflect = bc, lib.MG_K_FIXED, reflect
        for a in range(3):
            cfg.lo[a], cfg.hi[a] = lo, lo + 16.0
        return cfg
    assert lib.mg_workspace_size(cfg_for(lib.MG_BC_ROBIN, 7)) == lib.mg_workspace_size(cfg_for(lib.MG_BC_ROBIN, 0))
    for bad in (cfg_for(lib.MG_BC_PERIODIC, 1), cfg_for(lib.MG_BC_ROBIN, 8), cfg_for(lib.MG_BC_ROBIN, 2, lo=-8.0)):
        with pytest.raises(lib.MGError) as e:
            lib.mg_workspace_size(bad)
        assert e.value.status == lib.MG_ERR_INVALID_ARG


def test_extrapolating_face_validation(lib):
    """extrap needs a Robin box, a 6-bit mask, no lower face that is also a symmetry plane, and at
    least one face left Robin; it adds no workspace."""
    def cfg_for(bc, extrap, reflect=0):
        cfg = lib.mg_config_default()
        cfg.n[0] = cfg.n[1] = cfg.n[2] = 32
        cfg.bc, cfg.k_mode, cfg.extrap, cfg.reflect = bc, lib.MG_K_FIXED, extrap, reflect
        for a in range(3):
            cfg.lo[a], cfg.hi[a] = 0.0, 16.0
        return cfg
    assert lib.mg_workspace_size(cfg_for(lib.MG_BC_ROBIN, 0b000011)) == lib.mg_workspace_size(cfg_for(lib.MG_BC_ROBIN, 0))
    lib.mg_workspace_size(cfg_for(lib.MG_BC_ROBIN, 0b101010, reflect=1))   # one lower face stays Robin
    for bad in (cfg_for(lib.MG_BC_PERIODIC, 1), cfg_for(lib.MG_BC_ROBIN, 64), cfg_for(lib.MG_BC_ROBIN, -1),
                cfg_for(lib.MG_BC_ROBIN, 0b000001, reflect=1)):
        with pytest.raises(lib.MGError) as e:
            lib.mg_workspace_size(bad)
        assert e.value.status == lib.MG_ERR_INVALID_ARG
    for none_left in (cfg_for(lib.MG_BC_ROBIN, 63), cfg_for(lib.MG_BC_ROBIN, 0b101010, reflect=7)):
        with pytest.raises(lib.MGError) as e:
            lib.mg_workspace_size(none_left)
        assert e.value.status == lib.MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("field,value,status", [
    ("field_tol", -1e-10, 1), ("field_tol", float("nan"), 1), ("use_graph", 3, 1),
    ("order", 3, 1), ("bc", 7, 1), ("precision", 5, 1), ("levels", 6, 1), ("coarse_sweeps", 0, 1),
    ("nested", 2, 1), ("nested_min", 2, 1), ("nested_tol", -1.0, 1), ("tile_waves", -1, 1), ("tile_waves", 9, 1), ("field_est", 2, 1), ("k2_newton", 2, 1),
])
def test_invalid_configs_are_rejected_on_the_host(lib, field, value, status):
    cfg = lib.mg_config_default()
    setattr(cfg, field, value)
    with pytest.raises(lib.MGError) as e:
        lib.mg_workspace_size(cfg)
    assert e.value.status == status


def test_punctures_need_robin(lib):
    cfg = lib.mg_config_default()
    cfg.npunct = 1
    with pytest.raises(lib.MGError) as e:
        lib.mg_workspace_size(cfg)
    assert e.value.status == lib.MG_ERR_UNSUPPORTED


def test_status_strings(lib):
    L = lib.lib()
    assert L.mg_status_string(0) == b"MG_OK"
    assert L.mg_status_string(8) == b"MG_ERR_TIMEOUT"


def test_k2_newton_workspace(lib):
    """k2_newton adds the z solve's result and right-hand side (4N values of the inner type each) on
    periodic boxes with K from integrability, and nothing elsewhere."""
    def size(**over):
        cfg = lib.mg_config_default()
        for a in range(3):
            cfg.n[a] = 32
        for k, v in over.items():
            setattr(cfg, k, v)
        return lib.mg_workspace_size(cfg)
    base = size()
    assert size(k2_newton=1) - base >= 8 * 32 ** 3 * 4
    robin = dict(bc=lib.MG_BC_ROBIN, k_mode=lib.MG_K_FIXED)
    assert size(k2_newton=1, **robin) == size(**robin)
