"""The C ABI library loads on the host and exports every entry point include/b3d.h
declares; the binding defines the same names; struct layouts agree with the header.
No compute call here needs a GPU."""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "b3d.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:b3d_status|const char \*|int64_t|uint64_t)\s*(b3d_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_08715_gb300 import b3d
    return b3d.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["b3d_load_mesh", "b3d_set_scene", "b3d_render_batch", "b3d_score_batch", "b3d_enumerate_c2f",
                 "b3d_score_grad", "b3d_lse_resample", "b3d_sync", "b3d_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2312_08715_gb300 import b3d
    for name in _declared():
        assert hasattr(lib, name), name
        assert hasattr(b3d, name), f"binding lacks {name}"


def test_null_context_is_rejected_without_device_work(lib):
    assert lib.b3d_destroy(None) == -1
    assert lib.b3d_sync(None, None) == -1
    assert lib.b3d_score_batch(None, 0, 1, None, None, None, None) == -1
    assert lib.b3d_launch_count(None) == 0


def test_create_fails_cleanly_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2312_08715_gb300 import b3d
    with pytest.raises(b3d.B3DError) as e:
        b3d.b3d_create(0)
    assert e.value.status == b3d.B3D_EINVAL
    assert "device" in b3d.b3d_last_error(None)


def test_struct_layouts_match_the_header(tmp_path):
    from paper_2312_08715_gb300 import b3d
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "b3d.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(b3d_intrinsics), sizeof(b3d_lik_params), sizeof(b3d_stage), sizeof(b3d_c2f_schedule));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(b3d_c2f_schedule, stage), offsetof(b3d_c2f_schedule, n_particles),
         offsetof(b3d_c2f_schedule, seed), offsetof(b3d_c2f_schedule, grid_frame),
         offsetof(b3d_c2f_schedule, path_density));
  printf("%zu %zu\\n", offsetof(b3d_lik_params, volume), offsetof(b3d_lik_params, miss_mode));
  printf("%zu %zu\\n", sizeof(b3d_tuning), offsetof(b3d_tuning, high_occupancy));
  printf("%zu %zu %zu %zu %zu\\n", sizeof(b3d_score_item), sizeof(b3d_c2f_item), offsetof(b3d_c2f_item, particles_dev),
         offsetof(b3d_c2f_item, centre_dev), offsetof(b3d_c2f_item, map_dev));
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(b3d_server_config), offsetof(b3d_server_config, lik),
         offsetof(b3d_server_config, schedule), offsetof(b3d_server_config, tuning), sizeof(b3d_session_desc),
         offsetof(b3d_session_desc, grid_frame));
  printf("%zu %zu %zu %zu\\n", sizeof(b3d_frame_result), offsetof(b3d_frame_result, latency_ms),
         sizeof(b3d_server_stats), offsetof(b3d_server_stats, hbm_used));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [C.sizeof(b3d.b3d_intrinsics), C.sizeof(b3d.b3d_lik_params), C.sizeof(b3d.b3d_stage),
            C.sizeof(b3d.b3d_c2f_schedule),
            b3d.b3d_c2f_schedule.stage.offset, b3d.b3d_c2f_schedule.n_particles.offset,
            b3d.b3d_c2f_schedule.seed.offset, b3d.b3d_c2f_schedule.grid_frame.offset,
            b3d.b3d_c2f_schedule.path_density.offset,
            b3d.b3d_lik_params.volume.offset, b3d.b3d_lik_params.miss_mode.offset,
            C.sizeof(b3d.b3d_tuning), b3d.b3d_tuning.high_occupancy.offset,
            C.sizeof(b3d.b3d_score_item), C.sizeof(b3d.b3d_c2f_item), b3d.b3d_c2f_item.particles_dev.offset,
            b3d.b3d_c2f_item.centre_dev.offset, b3d.b3d_c2f_item.map_dev.offset,
            C.sizeof(b3d.b3d_server_config), b3d.b3d_server_config.lik.offset, b3d.b3d_server_config.schedule.offset,
            b3d.b3d_server_config.tuning.offset, C.sizeof(b3d.b3d_session_desc), b3d.b3d_session_desc.grid_frame.offset,
            C.sizeof(b3d.b3d_frame_result), b3d.b3d_frame_result.latency_ms.offset, C.sizeof(b3d.b3d_server_stats),
            b3d.b3d_server_stats.hbm_used.offset]
    assert got == want


def test_oracle_and_product_share_no_code():
    """The CUDA sources include nothing from oracle/ and the oracle nothing from the package."""
    csrc = os.path.join(ROOT, "paper_2312_08715_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower() or f.endswith(".md"), f
    pkg = os.path.join(ROOT, "paper_2312_08715_gb300")
    for f in sorted(os.listdir(pkg)):
        if not f.endswith(".py"):
            continue
        txt = open(os.path.join(pkg, f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f
    otxt_py = open(os.path.join(ROOT, "oracle", "oracle.py")).read()
    assert "paper_2312_08715_gb300" not in otxt_py.replace("paper_2312_08715_gb300.synth", "")
    otxt = open(os.path.join(ROOT, "oracle", "b3d_oracle.c")).read()
    assert "b3d.h" not in otxt and "b3d_internal" not in otxt



def test_binding_refuses_to_load_without_the_library(tmp_path):
    """No CPU fallback: with the compiled library absent (and no build asked for), loading the
    binding raises instead of handing out anything that computes on the host."""
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2312_08715_gb300 import b3d\n"
        "b3d._build.LIB = %r\n"
        "try:\n"
        "    b3d.load(build_if_missing=False)\n"
        "except ImportError as e:\n"
        "    print('refused' if 'not built' in str(e) else e)\n"
    ) % (ROOT, str(tmp_path / "missing" / "libb3d.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "refused", r.stdout + r.stderr
