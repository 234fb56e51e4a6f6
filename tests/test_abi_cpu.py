"""Host-side checks of the C ABI that need no GPU: the library loads,
exports every entry point include/gx.h declares, and rejects bad arguments
with GX_EINVAL before touching the device."""
import ctypes as C
import os
import re

import pytest

from paper_2306_07552_b300 import build as B
from paper_2306_07552_b300 import gx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return gx.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gx_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert sorted(gx.SYMBOLS) == names


def test_struct_sizes_match_header(tmp_path):
    """The ctypes mirrors against the C compiler's layout of include/gx.h."""
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"gx_robot": gx.GxRobot, "gx_scene_desc": gx.GxSceneDesc,
               "gx_object_mesh": gx.GxObjectMesh, "gx_config": gx.GxConfig,
               "gx_outputs": gx.GxOutputs, "gx_train_params": gx.GxTrainParams,
               "gx_tune_result": gx.GxTuneResult, "gx_scene_options": gx.GxSceneOptions}
    fields = {"gx_config": ["seed", "env_scene", "profile", "sdf_mode", "sdf_margin",
                            "broadphase", "render_robot", "heuristics", "static_store"],
              "gx_outputs": ["event", "reward", "task_obs", "success"],
              "gx_train_params": ["batch", "lr", "seed"]}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "gx.h"', "int main(void) {"]
    for name in structs:
        src.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in fields.get(name, []):
            src.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    src.append("  return 0;\n}")
    c = tmp_path / "sizes.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(root, "include"), "-o", str(exe), str(c)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f in fields.get(name, []):
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_null_arguments_are_rejected(L):
    out = C.c_void_p()
    assert L.gx_create(None, None, None, C.byref(out)) == gx.GX_EINVAL
    assert L.gx_scene_set_create(None, 0, None, C.byref(out)) == gx.GX_EINVAL
    assert L.gx_step(None, None, None, None) == gx.GX_EINVAL
    assert L.gx_reset(None, None, None) == gx.GX_EINVAL
    assert b"NULL" in L.gx_last_error(None) or L.gx_last_error(None)


def test_bad_scene_is_rejected_before_device_work(L):
    import numpy as np
    from paper_2306_07552_b300 import inputs as I
    s = I.room_scene(3, 300, n_furniture=2)
    s.tris = s.tris.copy()
    s.tris[0, 0] = 10 ** 6          # index out of range
    with pytest.raises(gx.GxError) as e:
        gx.SceneSet([s])
    assert e.value.status == gx.GX_EINVAL


def test_added_entry_points_validate_on_the_host(L):
    """The entry points added beside the step reject NULL or out-of-range
    arguments with GX_EINVAL before touching a device; the memory cap's
    counters are host state (no device needed)."""
    out = (C.c_int64 * 8)()
    assert L.gx_step_counters(None, out, 8) == gx.GX_EINVAL
    assert L.gx_apply_tune(None, None) == gx.GX_EINVAL
    assert L.gx_nsdf_train_steps(None, 0, None, 0, 1, None, None, None, None) == gx.GX_EINVAL
    assert L.gx_static_distance(None, 0, 0, None, 0, None, None) == gx.GX_EINVAL
    assert L.gx_scene_bytes(None, 0, None) == gx.GX_EINVAL
    opt = gx.GxSceneOptions(2, 1)           # options other than 0 / 1
    handle = C.c_void_p()
    assert L.gx_scene_set_create_ex(None, 1, None, C.byref(opt), C.byref(handle)) == gx.GX_EINVAL
    before = gx.device_memory_in_use()
    gx.set_device_memory_cap(1 << 20)
    assert gx.device_memory_in_use() == before
    gx.set_device_memory_cap(0)
