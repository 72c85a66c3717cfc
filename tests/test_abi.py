"""Host-only checks of the C ABI: the library loads, exports every function include/rmp.h
declares, its structs have the layout the header defines (checked against a C program
compiled from the header), and pure host calls (presets, status strings) behave.  No
call here touches a GPU."""
import ctypes as C
import json
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rmp.h")


@pytest.fixture(scope="module")
def rmp():
    from paper_2301_08068_gb300 import build, rmp as R
    build.build()
    R.lib()
    return R


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(rmp_[a-z_0-9]+)\s*\(",
                                 text, flags=re.M)))


def test_every_declared_function_is_exported(rmp):
    names = declared_functions()
    assert len(names) >= 12
    L = rmp.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(rmp.EXPORTS) == names


def test_struct_layouts_match_header(rmp, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "rmp.h"
#define O(T, f) printf("\\"%s.%s\\": %zu,\\n", #T, #f, offsetof(T, f))
int main(void) {
  printf("{\\n");
  printf("\\"rmp_params_t\\": %zu, \\"rmp_result_t\\": %zu, \\"rmp_ray_hit_t\\": %zu,\\n",
         sizeof(rmp_params_t), sizeof(rmp_result_t), sizeof(rmp_ray_hit_t));
  printf("\\"rmp_map_desc_t\\": %zu, \\"rmp_map_info_t\\": %zu, \\"rmp_launch_info_t\\": %zu,\\n",
         sizeof(rmp_map_desc_t), sizeof(rmp_map_info_t), sizeof(rmp_launch_info_t));
  O(rmp_params_t, max_range); O(rmp_params_t, halton_offset); O(rmp_params_t, flags);
  O(rmp_result_t, A); O(rmp_result_t, eig); O(rmp_result_t, n_rays); O(rmp_result_t, status);
  O(rmp_ray_hit_t, steps); O(rmp_ray_hit_t, d); O(rmp_ray_hit_t, status);
  O(rmp_map_desc_t, voxel_size); O(rmp_map_desc_t, dims); O(rmp_map_desc_t, n_blocks);
  O(rmp_map_desc_t, occ); O(rmp_map_desc_t, tsdf); O(rmp_map_info_t, device_bytes);
  O(rmp_map_info_t, layout); O(rmp_launch_info_t, ctas_per_sm); O(rmp_launch_info_t, ray_cells);
  printf("\\"rmp_server_config_t\\": %zu, \\"rmp_server_stats_t\\": %zu,\\n",
         sizeof(rmp_server_config_t), sizeof(rmp_server_stats_t));
  O(rmp_server_config_t, mem_budget_bytes); O(rmp_server_stats_t, max_inflight);
  printf("\\"rmp_rollout_params_t\\": %zu, \\"rmp_rollout_result_t\\": %zu,\\n",
         sizeof(rmp_rollout_params_t), sizeof(rmp_rollout_result_t));
  O(rmp_rollout_params_t, max_steps); O(rmp_rollout_result_t, status);
  O(rmp_rollout_result_t, smooth_segments);
  printf("\\"rmp_primitive_t\\": %zu,\\n", sizeof(rmp_primitive_t));
  O(rmp_primitive_t, center); O(rmp_primitive_t, size);
  printf("\\"end\\": 0}\\n");
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = json.loads(subprocess.check_output([str(exe)]))
    for T in ("rmp_params_t", "rmp_result_t", "rmp_ray_hit_t", "rmp_map_desc_t", "rmp_map_info_t",
              "rmp_launch_info_t", "rmp_server_config_t", "rmp_server_stats_t",
              "rmp_rollout_params_t", "rmp_rollout_result_t", "rmp_primitive_t"):
        assert C.sizeof(getattr(rmp, T)) == got[T], T
    for key, off in got.items():
        if "." in key:
            T, f = key.split(".")
            assert getattr(getattr(rmp, T), f).offset == off, key
    assert got["rmp_result_t"] == 144 and got["rmp_ray_hit_t"] == 24
    assert got["rmp_primitive_t"] == 56


def test_c_program_links_and_calls_host_functions(rmp, tmp_path):
    """The library is usable from plain C: a program compiled against include/rmp.h and
    linked with librmp.so calls the host-only entry points (no GPU needed)."""
    src = tmp_path / "use.c"
    src.write_text("""
#include <stdio.h>
#include <string.h>
#include "rmp.h"
int main(void) {
  rmp_params_t p;
  memset(&p, 0, sizeof(p));
  if (rmp_params_preset(RMP_PRESET_STATIC_MAP, &p) != RMP_OK) return 1;
  if (rmp_params_preset(7, &p) != RMP_ERR_INVALID_ARG) return 2;
  if (rmp_ctx_create(NULL, 0) != RMP_ERR_INVALID_ARG) return 3;
  if (strcmp(rmp_status_string(RMP_OK), "ok") != 0) return 4;
  printf("%.17g %.17g %zu %zu\\n", p.eta_rep, p.r, rmp_workspace_bytes(),
         rmp_batch_workspace_bytes(3, 1000));
  return 0;
}
""")
    exe = tmp_path / "use"
    lib = rmp.lib_path()
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe),
                           "-L", os.path.dirname(lib), "-lrmp",
                           "-Wl,-rpath," + os.path.dirname(lib)])
    out = subprocess.check_output([str(exe)], text=True).split()
    p = rmp.rmp_params_preset(rmp.RMP_PRESET_STATIC_MAP)
    assert float(out[0]) == p.eta_rep and float(out[1]) == p.r
    assert int(out[2]) == rmp.rmp_workspace_bytes()
    assert int(out[3]) == rmp.rmp_batch_workspace_bytes(3, 1000)


def test_presets_equal_table_one(rmp):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "table1_params.json")))
    for preset, col in ((rmp.RMP_PRESET_STATIC_MAP, "static_map"), (rmp.RMP_PRESET_LIDAR, "lidar")):
        p = rmp.rmp_params_preset(preset)
        for k in ("c", "eta_rep", "nu_rep", "eta_damp", "nu_damp", "r"):
            assert getattr(p, k) == gold[col][k], (col, k)
        assert p.halton_offset == 1 and p.flags == 0
    with pytest.raises(rmp.RmpError):
        rmp.rmp_params_preset(7)


def test_status_strings(rmp):
    assert rmp.rmp_status_string(0) == "ok"
    assert rmp.rmp_status_string(6) == "unknown map id"
    assert rmp.rmp_status_string(999) == "unknown status"


def test_workspace_size_is_fixed(rmp):
    """A 1024-byte header and one 80-byte partial slot per CTA of the largest grid."""
    assert rmp.rmp_workspace_bytes() == 1024 + 80 * 4096


def test_batch_workspace_size(rmp):
    """Header + states + tickets + one 80-byte partial per chunk (32 threads, up to 4
    segments per ray) and per group of 32 chunks, each region 256-byte aligned."""
    al = lambda x: (x + 255) // 256 * 256
    for B, mr in ((1, 1), (3, 1000), (256, 65536)):
        cps = (mr * 4 + 31) // 32
        gps = (cps + 31) // 32
        o = al(128)
        o = al(o + 80 * B)
        o = al(o + 4 * B)
        o = al(o + 4 * B * gps)
        o = al(o + 80 * B * cps)
        o = al(o + 80 * B * gps)
        assert rmp.rmp_batch_workspace_bytes(B, mr) == o
    assert rmp.rmp_batch_workspace_bytes(0, 10) == 0
    assert rmp.rmp_batch_workspace_bytes(10, 0) == 0
    assert rmp.rmp_batch_workspace_bytes(65537, 10) == 0


def test_null_arguments_rejected_without_gpu(rmp):
    L = rmp.lib()
    assert L.rmp_ctx_create(None, 0) == 1
    assert L.rmp_ctx_destroy(None) == 1
    assert L.rmp_map_release(None, 1) == 1
    assert L.rmp_raycast_eval(None, 1, None, None, 1, None, None, None, None, None) == 1
    assert L.rmp_scan_eval(None, None, 1, None, None, None, None, None, None) == 1
    assert L.rmp_raycast_eval_batch_async(None, 1, None, None, 1, 1, None, None, 0, None, None,
                                          None, None) == 1
    assert L.rmp_raycast_eval_batch(None, 1, None, None, 1, None, None, None) == 1
    assert L.rmp_batch_autotune(None, 1, None, None, 1, 1, None, None, 0, None, None, 1, None,
                                0) == 1
    assert L.rmp_server_create(None, None, None) == 1
    assert L.rmp_server_destroy(None) == 1
    assert L.rmp_server_submit(None, 1, None, None, 1, None, None) == 1
    assert L.rmp_server_poll(None, 1, None, None) == 1
    assert L.rmp_server_wait(None, 1, 0, None, None) == 1
    assert L.rmp_server_stats(None, None) == 1
    assert L.rmp_rollout(None, 1, None, 1, None, None, None, None) == 1
    assert L.rmp_combined_eval_batch_async(None, 1, None, None, 1, 1, None, None, 1.0, 1.0, 0,
                                           None, 0, None, None) == 1
    assert L.rmp_scan_pipeline_create(None, 1, 2, None) == 1
    assert L.rmp_scan_pipeline_destroy(None) == 1
    assert L.rmp_scan_pipeline_submit(None, None, 1, None, None, None, None) == 1
    assert L.rmp_scan_pipeline_wait(None, 1, None) == 1
    assert L.rmp_map_cell_distances(None, 1, None, None, None, 0) == 1
    cfg = rmp.rmp_server_config_default()
    assert (cfg.slots, cfg.max_batch_states, cfg.max_rays, cfg.mem_budget_bytes) == \
        (4, 256, 262144, 1 << 30)


def test_missing_library_fails_loudly(rmp, monkeypatch):
    """No fallback: when librmp.so is missing or stale and cannot be built, every use of the
    binding raises instead of computing anything some other way."""
    import paper_2301_08068_gb300.rmp as R
    saved = R._lib
    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R._build, "up_to_date", lambda: False)

    def no_toolchain():
        raise OSError("nvcc not found")
    monkeypatch.setattr(R._build, "build", no_toolchain)
    with pytest.raises(RuntimeError, match="could not be built"):
        R.lib()
    with pytest.raises(RuntimeError):
        R.rmp_params_preset(R.RMP_PRESET_STATIC_MAP)
    monkeypatch.setattr(R, "_lib", saved)


def test_context_without_gpu_is_an_error(rmp):
    """On a machine without a usable GPU the context cannot be created (status, no
    fallback)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rmp.RmpError):
        rmp.Context(0)


def test_fast_binding_marshalling():
    """The CPython extension of the synchronous calls (argument marshalling only) reaches
    the C ABI: a null context is refused with RMP_ERR_INVALID_ARG, malformed vectors raise,
    and its result decoding equals the ctypes structure's."""
    import numpy as np
    from paper_2301_08068_gb300 import rmp
    if not rmp.fast_binding():
        pytest.skip("CPython extension not built here (no Python headers)")
    bad = rmp.STATUS_CODES["RMP_ERR_INVALID_ARG"]
    for x, v in (([1.0, 2.0, 3.0], (0.0, 0.0, 0.0)), (np.zeros(3), np.ones(3, np.float32))):
        st, raw = rmp._fast.raycast_eval(None, 1, x, v, 64, 0, None, None, None)
        assert st == bad and len(raw) == 144
        st, raw = rmp._fast.scan_eval(None, None, 1, x, v, 0, None, None)
        assert st == bad and len(raw) == 144
    with pytest.raises(ValueError):
        rmp._fast.raycast_eval(None, 1, [1.0, 2.0], [0.0, 0.0, 0.0], 64, 0, None, None, None)
    r = rmp.rmp_result_t()
    for i in range(3):
        r.f[i], r.Af[i], r.eig[i] = 1.5 + i, -2.0 * i, 1e-3 * (i + 1)
    for i in range(6):
        r.A[i] = 0.25 * i
    r.n_rays, r.n_hits, r.n_active, r.rank, r.status = 65536, 1234, 77, 3, 0
    a, b = rmp.result_dict(r), rmp._result_from_raw(bytes(r))
    for k in ("f", "sumA", "sumAf", "eig"):
        assert np.array_equal(a[k], b[k])
    for k in ("n_rays", "n_hits", "n_active", "rank", "status"):
        assert a[k] == b[k]
