"""The C ABI: the library builds for sm_103a, loads, exports every call that
include/*.h declares, and validates descriptors on the host.  No GPU work."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

from conftest import ROOT
from paper_2305_13419_gb300 import build as tfbuild
from paper_2305_13419_gb300 import twofluid as tf
from paper_2305_13419_gb300 import workloads as W


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tf(?:64)?_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    return tf.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"tf_create", "tf_step", "tf_read_field", "tf_fit_q"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", tfbuild.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(tf(?:64)?_\w+)\b", out))
    assert names <= exported, names - exported
    for n in names:
        assert hasattr(lib, n)


def test_binding_covers_every_symbol():
    assert _declared() == set(tf.EXPORTS)


def test_build_targets_sm103a_only():
    gencodes = [tfbuild.NVCC_FLAGS[i + 1] for i, f in enumerate(tfbuild.NVCC_FLAGS) if f == "-gencode"]
    assert gencodes == ["arch=compute_103a,code=sm_103a"]


def _desc(**kw):
    w = W.cpw_small()
    args = dict(n=w.n, d=w.d, theta=1.0, bc=w.bc, cpml=w.cpml, courant=0.95)
    args.update(kw)
    return tf.make_desc(**args)


def test_workspace_size_scales_with_grid():
    a = tf.tf_workspace_size(_desc())
    b = tf.tf_workspace_size(_desc(n=(256, 64, 40)))
    assert a > 0 and b > a
    assert a % 256 == 0


@pytest.mark.parametrize("bad", [
    dict(n=(0, 4, 4)), dict(d=(-1.0, 1e-8, 1e-8)), dict(theta=0.3), dict(theta=1.5),
    dict(courant=0.0), dict(edge_rule=5), dict(max_probes=99),
])
def test_invalid_descriptors_rejected_on_host(bad):
    d = _desc(**bad)
    assert tf.tf_workspace_size(d) == 0
    h = C.c_void_p()
    rc = tf.load().tf_create(C.byref(d), C.c_void_p(256), C.c_size_t(1 << 30), C.byref(h))
    assert rc == tf.TF_EINVAL


def test_mur_only_on_z():
    d = _desc(bc=("mur", "periodic", "periodic"), cpml=(None, None, None))
    h = C.c_void_p()
    rc = tf.load().tf_create(C.byref(d), C.c_void_p(256), C.c_size_t(1 << 30), C.byref(h))
    assert rc == tf.TF_ENOTSUP


def test_cpml_thicker_than_half_axis_rejected():
    w = W.cpw_small()
    cp = W.default_cpml(w.n[0] // 2 + 1, w.d[0], 1e12)
    d = _desc(cpml=(cp, w.cpml[1], w.cpml[2]))
    assert tf.tf_workspace_size(d) == 0


def test_small_workspace_and_misaligned_pointer_rejected():
    d = _desc()
    need = tf.tf_workspace_size(d)
    h = C.c_void_p()
    L = tf.load()
    assert L.tf_create(C.byref(d), C.c_void_p(256), C.c_size_t(need - 1), C.byref(h)) == tf.TF_ENOMEM
    assert L.tf_create(C.byref(d), C.c_void_p(257), C.c_size_t(need), C.byref(h)) == tf.TF_EINVAL
    assert L.tf_create(C.byref(d), None, C.c_size_t(need), C.byref(h)) == tf.TF_EINVAL


def test_over_courant_rejected():
    d = _desc(courant=1.2)
    h = C.c_void_p()
    assert tf.load().tf_create(C.byref(d), C.c_void_p(256), C.c_size_t(1 << 34), C.byref(h)) == tf.TF_EUNSTABLE


def test_null_handle_calls_fail_cleanly():
    L = tf.load()
    assert L.tf_step(None, 1) == tf.TF_EINVAL
    assert L.tf_sync(None) == tf.TF_EINVAL
    assert L.tf_destroy(None) == tf.TF_EINVAL
    assert L.tf_set_two_step(None, 1) == tf.TF_EINVAL
    assert L.tf_set_wait_limit(None, 0) == tf.TF_EINVAL
    assert L.tf_set_item_planes(None, 8) == tf.TF_EINVAL
    assert tf.tf_strerror(tf.TF_ENONFINITE) == "non-finite field value"


def _size_and_create(n, bc=("periodic", "periodic", "pec")):
    d = _desc(n=n, bc=bc, cpml=(None, None, None))
    h = C.c_void_p()
    return tf.tf_workspace_size(d), d, h


def test_largest_descriptor_grids_accepted_one_past_rejected():
    """Work-item descriptors carry 20 bits of tile index and 20 bits of
    plane: a grid with exactly 2^20 storage planes along z, or exactly 2^20
    32 x 16 tiles, is accepted (its workspace is sized; nothing is
    allocated), one plane or one tile column more is refused on the host
    (TF_ENOTSUP), and more than 2^40 storage points is TF_EINVAL."""
    L = tf.load()
    size, _, _ = _size_and_create((4, 4, (1 << 20) - 1))          # 2^20 storage planes (walled z)
    assert size > 0
    size, d, h = _size_and_create((4, 4, 1 << 20))
    assert size == 0
    assert L.tf_create(C.byref(d), C.c_void_p(256), C.c_size_t(1 << 30), C.byref(h)) == tf.TF_ENOTSUP
    # 32768 x 16384 storage columns: 1024 x 1024 tiles
    size, _, _ = _size_and_create((32767, 16383, 1), bc=("pec", "pec", "pec"))
    assert size > 0
    size, d, h = _size_and_create((32768, 16383, 1), bc=("pec", "pec", "pec"))
    assert size == 0
    assert L.tf_create(C.byref(d), C.c_void_p(256), C.c_size_t(1 << 30), C.byref(h)) == tf.TF_ENOTSUP
    size, d, h = _size_and_create((1 << 14, 1 << 14, 1 << 13), bc=("periodic", "periodic", "periodic"))
    assert size == 0
    assert L.tf_create(C.byref(d), C.c_void_p(256), C.c_size_t(1 << 30), C.byref(h)) == tf.TF_EINVAL
