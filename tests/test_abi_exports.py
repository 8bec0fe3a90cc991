"""The C-ABI library builds, loads and exports every entry point include/aco.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aco.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aco_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["aco_create_instance", "aco_build_candidates", "aco_construct_tours", "aco_update_pheromone",
                     "aco_tour_lengths", "aco_destroy_instance", "aco_build_candidates_noalloc"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1709_03187_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_has_every_entry_point():
    import paper_1709_03187_gb300 as pkg

    for n in _declared():
        if n in ("aco_status_string", "aco_last_error", "aco_batch_last_error", "aco_mlp_last_error"):
            continue
        assert hasattr(pkg, n), n


def test_struct_layouts_match_ctypes(tmp_path):
    """sizeof/offsetof of the ABI structs as a C compiler sees the header == the binding's."""
    from paper_1709_03187_gb300._ffi import Params, Stats

    prog = tmp_path / "sz.c"
    prog.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "aco.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(aco_params), sizeof(aco_stats),'
                    ' offsetof(aco_params, seed), offsetof(aco_params, fallback), offsetof(aco_stats, gbest));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out == [ctypes.sizeof(Params), ctypes.sizeof(Stats), Params.seed.offset, Params.fallback.offset,
                   Stats.gbest.offset]


def test_status_strings_without_gpu():
    from paper_1709_03187_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.aco_status_string.restype = ctypes.c_char_p
    assert lib.aco_status_string(0) == b"ok"
    assert lib.aco_status_string(1) == b"invalid argument"


def test_device_byte_limit_gives_oom_before_any_device_call():
    """ACO_DEVICE_BYTES_LIMIT below an instance's buffers: aco_create_instance returns ACO_ERR_OOM
    from its dry run, before it touches the device (so this runs without a GPU)."""
    import sys

    code = r'''
import ctypes, sys
sys.path.insert(0, sys.argv[1])
from paper_1709_03187_gb300 import build
from paper_1709_03187_gb300._ffi import Params
lib = ctypes.CDLL(build.build())
lib.aco_last_error.restype = ctypes.c_char_p
p = Params(1, 200000, 1024, 16, 1.0, 2.0, 0.1, 1.0, 0.01, 1.0, 3, 0, 0)
h = ctypes.c_void_p()
dummy = ctypes.c_void_p(0x1000)
st = lib.aco_create_instance(dummy, ctypes.byref(p), None, ctypes.byref(h))
print(st, lib.aco_last_error(None).decode())
'''
    env = dict(os.environ, ACO_DEVICE_BYTES_LIMIT="1000000")
    r = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    status, msg = r.stdout.split(" ", 1)
    assert int(status) == 2 and "ACO_DEVICE_BYTES_LIMIT" in msg  # ACO_ERR_OOM


def test_invalid_parameters_are_refused_before_any_device_call():
    """aco_create_instance checks its arguments before it touches the device, so each refusal
    (ACO_ERR_INVALID_ARG with the reason in aco_last_error) shows without a GPU."""
    import sys

    code = r'''
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
from paper_1709_03187_gb300 import build
from paper_1709_03187_gb300._ffi import Params
lib = ctypes.CDLL(build.build())
lib.aco_last_error.restype = ctypes.c_char_p
# (mode, n, m, k, alpha, beta, rho, tau0, max_mod_frac, p_partial, seed, fallback, selection)
ok = (1, 1000, 64, 16, 1.0, 2.0, 0.1, 1.0, 0.1, 1.0, 3, 0, 0)
cases = {
    "mode": dict(mode=7),
    "n < 3": dict(n=2),
    "m must be in [1, 16384]": dict(m=0),
    "k must be in [1, min(32, n-1)]": dict(k=33),
    "alpha, beta must be finite and >= 0": dict(alpha=float("nan")),
    "tau0 must be > 0": dict(tau0=0.0),
    "max_mod_frac in (0,1]": dict(max_mod_frac=0.0),
    "p_partial in [0,1]": dict(p_partial=1.5),
    "fallback must be 0 or 1": dict(fallback=2),
    "selection must be 0 or 1": dict(selection=3),
    "beta must be > 0 with candidate lists": dict(beta=0.0),
    "Independent Roulette needs candidate lists (LBEST mode)": dict(mode=0, k=0, selection=1),
    "DENSE mode supports n <= 8192": dict(mode=0, k=0, n=9000),
    "n too large for the visited bitset": dict(n=2000000, m=8),
    "n*m must be < 2^31": dict(n=1000000, m=4096),
}
names = ["mode", "n", "m", "k", "alpha", "beta", "rho", "tau0", "max_mod_frac", "p_partial", "seed",
         "fallback", "selection"]
out = {}
for why, change in cases.items():
    v = dict(zip(names, ok))
    v.update(change)
    p = Params(*[v[k] for k in names])
    h = ctypes.c_void_p()
    st = lib.aco_create_instance(ctypes.c_void_p(0x1000), ctypes.byref(p), None, ctypes.byref(h))
    out[why] = [st, lib.aco_last_error(None).decode(), h.value]
p = Params(*ok)
h = ctypes.c_void_p()
st = lib.aco_create_instance(ctypes.c_void_p(0x1004), ctypes.byref(p), None, ctypes.byref(h))
out["xy_dev not 8-byte aligned"] = [st, lib.aco_last_error(None).decode(), h.value]
print(json.dumps(out))
'''
    r = subprocess.run([sys.executable, "-c", code, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    import json

    out = json.loads(r.stdout.strip().splitlines()[-1])
    for why, (status, msg, handle) in out.items():
        assert status == 1, (why, status, msg)  # ACO_ERR_INVALID_ARG
        assert msg == why, (why, msg)
        assert handle is None, why


def test_noalloc_refusals_before_any_device_call():
    """aco_build_candidates_noalloc checks its pointers and sizes before any CUDA call: null or
    misaligned buffers, n outside [2, 65,536] and k outside [1, min(32, n - 1)] give
    ACO_ERR_INVALID_ARG without a GPU."""
    from paper_1709_03187_gb300 import build

    lib = ctypes.CDLL(build.build())
    f = lib.aco_build_candidates_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    xy, out = 0x1000, 0x2000  # never dereferenced: every case below is refused first
    cases = [(None, 100, 8, out), (xy, 100, 8, None), (0x1004, 100, 8, out), (xy, 100, 8, 0x2002),
             (xy, 1, 1, out), (xy, 65_537, 8, out), (xy, 100, 0, out), (xy, 100, 33, out), (xy, 10, 10, out)]
    for c in cases:
        assert f(c[0], c[1], c[2], c[3], None) == 1, c  # ACO_ERR_INVALID_ARG


def test_every_entry_point_refuses_a_null_handle_without_a_gpu():
    """Every call on an instance, a batch or a network checks its handle first: a null handle gives
    ACO_ERR_INVALID_ARG (and the destroy calls do nothing), so a caller's mistake there never
    reaches the device."""
    import sys

    code = r'''
import ctypes as C, sys
sys.path.insert(0, sys.argv[1])
from paper_1709_03187_gb300 import build
lib = C.CDLL(build.build())
P, I32, I64, D, F = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_float
sig = {
    "aco_build_candidates": [P, P], "aco_construct_tours": [P, I32, P, P], "aco_update_pheromone": [P],
    "aco_tour_lengths": [P, P, I32, P], "aco_get_state": [P, P, P, P], "aco_set_state": [P, P, P],
    "aco_get_stats": [P, P], "aco_step_probs": [P, I32, P, P, P], "aco_set_max_mod_frac": [P, D],
    "aco_set_p_partial": [P, D], "aco_set_local_search": [P, D, I32], "aco_set_async_share": [P, I32],
    "aco_set_ant_range": [P, I32, I32], "aco_export_commits": [P, P, I64, P],
    "aco_import_commits": [P, P, I32, I64], "aco_batch_build_candidates": [P],
    "aco_batch_run": [P, I32, I32, I32], "aco_batch_get_state": [P, P, P], "aco_batch_get_best": [P, P],
    "aco_batch_schedule": [P, P, P, P, P, P], "aco_batch_set_schedule": [P, I32],
    "aco_batch_set_wait_limit": [P, D], "aco_batch_instance": [P, I32, P], "aco_mlp_get_weights": [P, P],
    "aco_mlp_forward": [P, P, I64, P, P, F], "aco_mlp_backward": [P, P, P, I32, I32, F, P, P],
    "aco_mlp_adam": [P, P, F], "aco_mlp_train": [P, P, P, I32, I32, I32, I32, F, P],
    "aco_edge_features": [P, I32, P], "aco_tour_labels": [P, P], "aco_set_edge_scores": [P, P],
}
bad = []
for name, args in sig.items():
    f = getattr(lib, name)
    f.argtypes = args
    f.restype = C.c_int
    vals = [None if a is P else a(0) for a in args]
    st = f(*vals)
    if st != 1:
        bad.append((name, st))
for name in ("aco_destroy_instance", "aco_batch_destroy", "aco_mlp_destroy"):
    f = getattr(lib, name)
    f.argtypes = [P]
    f.restype = None
    f(None)
print("bad", bad)
'''
    r = subprocess.run([sys.executable, "-c", code, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().splitlines()[-1] == "bad []", r.stdout
