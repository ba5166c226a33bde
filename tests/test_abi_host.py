"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

import paper_2304_01772_gb300 as sm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EINVAL = -1


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "spinmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spin_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = sm.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert lib.spin_version() == 2
    assert lib.spin_mlp_param_count() == 3 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2


def test_binding_covers_the_abi():
    assert set(declared_symbols()) == set(sm._SIGS)


def _init(model, descs, cpm=None):
    arr = (sm.LatticeDesc * len(descs))(*descs)
    ctx = ctypes.c_void_p()
    rc = sm.lib().spin_init(ctypes.byref(ctx), model, 0, len(descs), arr,
                            ctypes.byref(cpm) if cpm else None, ctypes.c_void_p(16), 0, 0, None)
    return rc, ctx


@pytest.mark.parametrize("desc,model", [
    (sm.LatticeDesc(63, 2, 0.4, 1.0, 0.0, 0, 0.0, 0, 0), sm.SPIN_ISING),          # odd L
    (sm.LatticeDesc(2, 2, 0.4, 1.0, 0.0, 0, 0.0, 0, 0), sm.SPIN_ISING),           # too small
    (sm.LatticeDesc(64, 2, float("nan"), 1.0, 0.0, 0, 0.0, 0, 0), sm.SPIN_ISING),  # NaN beta
    (sm.LatticeDesc(64, 2, -0.1, 1.0, 0.0, 0, 0.0, 0, 0), sm.SPIN_ISING),         # negative beta
    (sm.LatticeDesc(64, 1, 0.4, 1.0, 0.0, 0, 0.0, 0, 0), sm.SPIN_POTTS),          # q < 2
    (sm.LatticeDesc(64, 256, 0.4, 1.0, 0.0, 0, 0.0, 0, 0), sm.SPIN_POTTS),        # q > 255
    (sm.LatticeDesc(64, 3, 0.4, 1.0, 0.1, 0, 0.0, 0, 0), sm.SPIN_POTTS),          # Potts with a field
    (sm.LatticeDesc(64, 2, 0.4, 1.0, 0.0, 1, 0.0, 0, 0), sm.SPIN_ISING),          # reserved != 0
])
def test_invalid_lattices_rejected(desc, model):
    rc, ctx = _init(model, [desc])
    assert rc == -1 and not ctx.value


def test_overlapping_lattices_rejected():
    rc, _ = _init(sm.SPIN_ISING, [sm.LatticeDesc(16, 2, 0.4, 1.0, 0.0, 0, 0.0, 0, 0),
                                  sm.LatticeDesc(16, 2, 0.4, 1.0, 0.0, 0, 0.0, 0, 100)])
    assert rc == -1


def test_cpm_parameter_checks():
    J = (ctypes.c_int32 * 9)(0, 16, 16, 16, 2, 11, 16, 12, 14)   # not symmetric
    cp = sm.CpmParams(3, 1, 400, 10, J, None, 10.0, 4, 5, 0)
    rc, _ = _init(sm.SPIN_CPM, [sm.LatticeDesc(64, 2, 0.0, 0.0, 0.0, 0, 0.0, 0, 0)], cp)
    assert rc == -1
    Jok = (ctypes.c_int32 * 9)(0, 16, 16, 16, 2, 11, 16, 11, 14)
    cp = sm.CpmParams(3, 1, 400, 10, Jok, None, 10.0, 4, 5, 0)
    rc, _ = _init(sm.SPIN_CPM, [sm.LatticeDesc(66, 2, 0.0, 0.0, 0.0, 0, 0.0, 0, 0)], cp)   # L % 4 != 0
    assert rc == -1
    rc, _ = _init(sm.SPIN_ISING, [sm.LatticeDesc(64, 2, 0.4, 1.0, 0.0, 0, 0.0, 0, 0)], cp)  # cpm for Ising
    assert rc == -1


def test_pack_offsets_alignment():
    off, total = sm.pack_offsets([32, 10, 2048, 4], elem=1, align=256)
    assert all(o % 256 == 0 for o in off)
    assert total == off[-1] + 16
    off4, _ = sm.pack_offsets([8, 8], elem=4, align=256)
    assert off4 == [0, 64]


def test_dmc_entry_points_reject_invalid_arguments_on_the_host():
    lib = sm.lib()
    assert lib.spin_dmc_tape_floats(4, 16, 3) == 4 * 2 * 3 * 16 * 16 // 2
    for B, L, n in [(0, 16, 1), (1, 12, 1), (1, 72, 1), (1, 4, 1), (1, 16, 0)]:
        assert lib.spin_dmc_tape_floats(B, L, n) == EINVAL
    buf = ctypes.c_void_p(256)   # aligned but never dereferenced: rejected first
    bad_geom = lib.spin_dmc_forward(1, 1, 12, 0.5, 0.0, 1.0, buf, buf, 0, 1, buf, None)
    bad_beta = lib.spin_dmc_forward(1, 1, 16, float("nan"), 0.0, 1.0, buf, buf, 0, 1, buf, None)
    misaligned = lib.spin_dmc_forward(1, 1, 16, 0.5, 0.0, 1.0, ctypes.c_void_p(260), buf, 0, 1, buf, None)
    null_ptr = lib.spin_dmc_backward(1, 1, 16, 0.5, 0.0, 1.0, buf, buf, buf, 0, 1, None, buf, None)
    assert bad_geom == bad_beta == misaligned == null_ptr == EINVAL
    assert lib.spin_dmc_discretize(-1, buf, None) == EINVAL
    assert lib.spin_dmc_discretize(0, None, None) == 0
    assert lib.spin_dmc_loss(0, 16, buf, buf, buf, buf, None) == EINVAL


def test_cpm_batch_entry_points_reject_invalid_arguments_on_the_host():
    lib = sm.lib()
    J = (ctypes.c_int32 * 9)(0, 16, 16, 16, 2, 11, 16, 11, 14)
    good = sm.CpmParams(3, 1, 25, 36, J, None, 8.0, 5, 6, 0)
    assert lib.spin_cpm_batch_workspace_bytes(ctypes.byref(good)) > 256
    buf = ctypes.c_void_p(256)
    assert lib.spin_cpm_batch_run(1, 4, 66, ctypes.byref(good), buf, buf, buf, 0, 1, None, buf, None) == EINVAL
    assert lib.spin_cpm_batch_run(1, 4, 64, ctypes.byref(good), buf, buf, buf, 0, 0, None, buf, None) == EINVAL
    assert lib.spin_cpm_batch_run(1, 4, 64, ctypes.byref(good), buf, buf, buf, 0, 1, None,
                                  ctypes.c_void_p(260), None) == EINVAL
    asym = (ctypes.c_int32 * 9)(0, 16, 15, 16, 2, 11, 16, 11, 14)
    bad = sm.CpmParams(3, 1, 25, 36, asym, None, 8.0, 5, 6, 0)
    assert lib.spin_cpm_batch_init(1, 4, 64, ctypes.byref(bad), buf, buf, buf, None) == EINVAL
    big = sm.CpmParams(3, 1, 25, 36, J, None, 8.0, 20, 6, 0)   # 6 x 20 > 64: does not fit
    assert lib.spin_cpm_batch_init(1, 4, 64, ctypes.byref(big), buf, buf, buf, None) == EINVAL


@pytest.mark.parametrize("desc,model", [
    (sm.LatticeDesc(48, 2, 0.4, 1.0, 0.0, 3, 0.0, 0, 0), sm.SPIN_ISING),   # unknown geometry
    (sm.LatticeDesc(48, 3, 0.4, 1.0, 0.0, 2, 0.5, 0, 0), sm.SPIN_POTTS),   # second neighbours are Ising only
    (sm.LatticeDesc(48, 2, 0.4, 1.0, 0.0, 0, 0.5, 0, 0), sm.SPIN_ISING),   # J2 without second neighbours
    (sm.LatticeDesc(48, 2, 0.4, 1.0, 0.0, 2, float("inf"), 0, 0), sm.SPIN_ISING),   # non-finite J2
    (sm.LatticeDesc(64, 2, 0.4, 1.0, 0.0, 1, 0.0, 0, 0), sm.SPIN_ISING),   # triangular needs L % 6 == 0
    (sm.LatticeDesc(48, 3, 0.4, 1.0, 0.0, 1, 0.0, 0, 0), sm.SPIN_POTTS),   # triangular is Ising only
])
def test_geometry_is_validated(desc, model):
    rc, _ = _init(model, [desc])
    assert rc == EINVAL


def test_second_neighbour_lattices_do_not_share_a_context():
    rc, _ = _init(sm.SPIN_ISING, [sm.LatticeDesc(16, 2, 0.4, 1.0, 0.0, 2, 0.5, 0, 0),
                                  sm.LatticeDesc(16, 2, 0.4, 1.0, 0.0, 0, 0.0, 0, 256)])
    assert rc == EINVAL
    rc, _ = _init(sm.SPIN_ISING, [sm.LatticeDesc(18, 2, 0.4, 1.0, 0.0, 1, 0.0, 0, 0),
                                  sm.LatticeDesc(16, 2, 0.4, 1.0, 0.0, 2, 0.5, 0, 512)])
    assert rc == EINVAL


def test_lattice_desc_layout_matches_the_header():
    assert ctypes.sizeof(sm.LatticeDesc) == 40
    assert sm.LatticeDesc.J2.offset == 24 and sm.LatticeDesc.spin_offset.offset == 32


def test_barrier_selftest_rejects_invalid_arguments_on_the_host():
    lib = sm.lib()
    for blocks, missing, rounds in [(0, 0, 1), (4, -1, 1), (4, 5, 1), (4, 0, 0)]:
        assert lib.spin_barrier_selftest(blocks, missing, rounds, None) == EINVAL


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structs have the C layout of include/spinmc.h (sizes and
    field offsets as gcc lays them out)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    fields = {"spin_lattice_desc": [f for f, _ in sm.LatticeDesc._fields_],
              "spin_cpm_params": [f if f != "lambda_" else "lambda" for f, _ in sm.CpmParams._fields_]}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "spinmc.h"', "int main(void) {"]
    for st, fs in fields.items():
        src.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            src.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for st, cls in (("spin_lattice_desc", sm.LatticeDesc), ("spin_cpm_params", sm.CpmParams)):
        assert int(got[st]) == ctypes.sizeof(cls), st
        for (f, _), cf in zip(cls._fields_, fields[st]):
            assert int(got[f"{st}.{cf}"]) == getattr(cls, f).offset, (st, f)


def test_bounds_checked_variant_builds_and_exports_the_abi():
    """The SPIN_CHECK variant (kernels with no-trap bounds checks) builds and
    exports every declared symbol, spin_check_status included."""
    from paper_2304_01772_gb300 import build
    lib = ctypes.CDLL(build.build(variant="check"))
    for n in declared_symbols():
        assert hasattr(lib, n), n
