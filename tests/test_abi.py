"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/mabd.h declares, the binding's struct mirrors match
the C layout, and argument validation returns status codes."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mabd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2603_08079_gb300 import mabd
    return mabd.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(mabd_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2603_08079_gb300 import mabd
    assert set(mabd.EXPORTS) <= set(names)


def test_struct_layout_matches_header(tmp_path):
    from paper_2603_08079_gb300 import mabd
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "mabd.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(mabd_body_desc), sizeof(mabd_joint_desc),
         sizeof(mabd_config), sizeof(mabd_step_stats), sizeof(mabd_info));
  printf("%zu %zu %zu %zu\n", offsetof(mabd_body_desc, q), offsetof(mabd_body_desc, fixed),
         offsetof(mabd_joint_desc, body_a), offsetof(mabd_joint_desc, axis_len));
  printf("%zu %zu %zu\n", offsetof(mabd_config, stream), offsetof(mabd_config, dev_alloc),
         offsetof(mabd_config, residual_rhs));
  printf("%zu %zu\n", offsetof(mabd_joint_desc, ref_a), offsetof(mabd_joint_desc, ref_b));
  printf("%zu %zu %zu %zu\n", offsetof(mabd_config, rotation_mode), offsetof(mabd_config, jacobian_mode),
         offsetof(mabd_info, rotation_mode), offsetof(mabd_info, jacobian_mode));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    vals = [int(v) for v in out]
    assert vals[0] == mabd.BODY_DTYPE.itemsize
    assert vals[1] == mabd.JOINT_DTYPE.itemsize
    assert vals[2] == C.sizeof(mabd.Config)
    assert vals[3] == C.sizeof(mabd.StepStats)
    assert vals[4] == C.sizeof(mabd.Info)
    assert vals[5] == mabd.BODY_DTYPE.fields["q"][1]
    assert vals[6] == mabd.BODY_DTYPE.fields["fixed"][1]
    assert vals[7] == mabd.JOINT_DTYPE.fields["body_a"][1]
    assert vals[8] == mabd.JOINT_DTYPE.fields["axis_len"][1]
    assert vals[9] == mabd.Config.stream.offset
    assert vals[10] == mabd.Config.dev_alloc.offset
    assert vals[11] == mabd.Config.residual_rhs.offset
    assert vals[12] == mabd.JOINT_DTYPE.fields["ref_a"][1]
    assert vals[13] == mabd.JOINT_DTYPE.fields["ref_b"][1]
    assert vals[14:18] == [mabd.Config.rotation_mode.offset, mabd.Config.jacobian_mode.offset,
                           mabd.Info.rotation_mode.offset, mabd.Info.jacobian_mode.offset]


def test_config_defaults_and_status_strings(lib):
    from paper_2603_08079_gb300 import mabd
    cfg = mabd.Config()
    lib.mabd_config_default(C.byref(cfg))
    assert cfg.h == 1e-2 and cfg.gravity[2] == -9.8 and cfg.residual_rhs == 1
    assert cfg.pcg_max_iters > 0 and cfg.pcg_rtol > 0
    assert cfg.rotation_mode == 0 and cfg.jacobian_mode == 0  # polar R, frozen frame
    for code in range(11):
        assert lib.mabd_status_string(code).decode() != "unknown status"


def test_argument_validation_without_a_device(lib):
    from paper_2603_08079_gb300 import mabd
    out = C.c_void_p()
    assert lib.mabd_create(None, C.byref(out)) == 1
    cfg = mabd.Config()
    lib.mabd_config_default(C.byref(cfg))
    cfg.h = -1.0
    assert lib.mabd_create(C.byref(cfg), C.byref(out)) == 1
    cfg.h = 1e-2
    cfg.solver = 9
    assert lib.mabd_create(C.byref(cfg), C.byref(out)) == 1
    cfg.solver = 0
    for field in ("rotation_mode", "jacobian_mode"):
        setattr(cfg, field, 2)
        assert lib.mabd_create(C.byref(cfg), C.byref(out)) == 1
        setattr(cfg, field, 0)
    # calls on a NULL context are rejected, not dereferenced
    assert lib.mabd_step(None, 1, None) == 1
    assert lib.mabd_prefactor(None) == 1
    assert lib.mabd_get_state(None, None, None) == 1
    assert lib.mabd_destroy(None) == 1


def test_scene_marshalling_roundtrip():
    from paper_2603_08079_gb300 import mabd, scenes
    sc = scenes.random_small("graph", 7, seed=1)
    b = mabd.body_array(sc)
    j = mabd.joint_array(sc)
    np.testing.assert_array_equal(b["q"], sc["q"])
    np.testing.assert_array_equal(b["second_moment"], sc["second_moment"])
    np.testing.assert_array_equal(j["body_b"], sc["body_b"])
    np.testing.assert_array_equal(j["type"], sc["jtype"])
    np.testing.assert_array_equal(j["axis_len"], sc["axis_len"])
