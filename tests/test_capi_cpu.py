"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point include/veckm.h declares, validates arguments on
the host, and its SplitMix64 + Box-Muller draw of the frequencies matches the
input generator's independent implementation of the same published
definition."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2504_19417_gb300 import synth
from paper_2504_19417_gb300 import veckm as vk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "veckm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(veckm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = vk.lib()
    names = _declared()
    assert "veckm_create" in names and "veckm_predict" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(vk.EXPORTS)


def test_checks_reader_is_refused_by_the_normal_build():
    # the bounds-checked build is a separate library; this one has no checks
    with pytest.raises(vk.VeckmError) as ei:
        vk.debug_checks()
    assert ei.value.status == vk.VECKM_EUNSUPPORTED


def test_normals_match_generator():
    for seed in (0, 1, 2, 12345):
        a = vk.normals(seed, 257)
        b = synth.normals(seed, 257)
        assert np.max(np.abs(a - b)) < 1e-12


def _cfg(**kw):
    w = synth.mlp_weights(64)
    base = dict(width=64, height=48, D=64, dx=10, dy=10, hidden=128, dt_us=16000, t_span_us=0,
                sigma2=25.0, freq_seed=0, flags=0)
    base.update(kw)
    c = vk._Config(**base)
    keep = [w.W1, w.b1, w.W2, w.b2]
    c.h_W1, c.h_b1, c.h_W2, c.h_b2 = (a.ctypes.data_as(C.c_void_p) for a in keep)
    return c, keep


@pytest.mark.parametrize("bad", [dict(width=0), dict(height=40000), dict(D=96), dict(D=32),
                                 dict(dx=-1), dict(dy=65), dict(hidden=64), dict(dt_us=0),
                                 dict(flags=3), dict(flags=8), dict(t_span_us=1 << 33),
                                 dict(D=256, flags=1), dict(flags=4)])
def test_create_rejects_bad_config_on_host(bad):
    c, keep = _cfg(**bad)
    h = C.c_void_p()
    st = vk.lib().veckm_create(C.byref(h), C.byref(c))
    assert st in (vk.VECKM_EINVAL, vk.VECKM_EUNSUPPORTED)
    assert not h.value
    assert vk.lib().veckm_last_error()


def test_create_rejects_null_arguments():
    h = C.c_void_p()
    assert vk.lib().veckm_create(C.byref(h), None) == vk.VECKM_EINVAL
    c, keep = _cfg()
    c.h_W1 = None
    assert vk.lib().veckm_create(C.byref(h), C.byref(c)) == vk.VECKM_EINVAL


def test_calls_on_null_context_are_rejected():
    L = vk.lib()
    assert L.veckm_encode(None, None, None, None, 0, 0, None, 0, None, None) == vk.VECKM_EINVAL
    assert L.veckm_predict(None, None, None, None, 0, 0, None, 0, None, None) == vk.VECKM_EINVAL
    assert L.veckm_sync_status(None, None) == vk.VECKM_EINVAL
    L.veckm_destroy(None)  # NULL-safe


def test_error_path_hooks_validate_on_host():
    L = vk.lib()
    assert L.veckm_set_injection(None, vk.INJECT_HEAD_STALL) == vk.VECKM_EINVAL
    assert L.veckm_set_wait_limit(None, 1000) == vk.VECKM_EINVAL
    # the allocation counter: reset, no allocation happens on a rejected
    # create (host-side checks come first), reset again
    vk.debug_fail_alloc(-1)
    c, keep = _cfg(width=0)
    h = C.c_void_p()
    assert L.veckm_create(C.byref(h), C.byref(c)) == vk.VECKM_EINVAL
    assert vk.debug_fail_alloc(-1) == 0


def test_tensor_core_head_rejects_weights_beyond_fp16_range():
    # |h_j| <= sum_c |W1_jc| + |b1_j| must stay inside the FP16 range of the
    # second layer's operand
    w = synth.mlp_weights(64)
    W1 = w.W1.copy()
    W1[5, :] = 1000.0
    c, keep = _cfg(flags=vk.MLP_FP16)
    keep.append(W1)
    c.h_W1 = W1.ctypes.data_as(C.c_void_p)
    h = C.c_void_p()
    assert vk.lib().veckm_create(C.byref(h), C.byref(c)) == vk.VECKM_EUNSUPPORTED
    assert not h.value
    assert b"FP16" in vk.lib().veckm_last_error()


def test_server_rejects_bad_window_limits_on_host():
    c, keep = _cfg()
    for bad in (dict(window_us=-1), dict(window_capacity=-5),
                dict(window_capacity=(1 << 30) + 1), dict(arena_bytes=-1)):
        sc = vk._ServerConfig(model=c, **bad)
        h = C.c_void_p()
        assert vk.lib().veckm_server_create(C.byref(sc), C.byref(h)) == vk.VECKM_EINVAL
        assert not h.value
