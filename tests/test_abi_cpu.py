"""C ABI checks that need no GPU: the library loads, exports every function that
include/*.h declares, and rejects bad arguments on the host before touching CUDA."""
import ctypes
import glob
import os
import re

import pytest

from paper_2607_10280_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_10280_b300 import build
    build.build()
    return _lib.lib()


def test_header_declares_the_four_path_calls():
    names = declared_functions()
    for fn in ("mps_create_batch", "mps_apply_circuit", "mps_pauli_cache", "ano_features"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for fn in names:
        assert hasattr(lib, fn), fn
    for fn in names:
        assert fn in _lib.SIGNATURES, f"binding lacks {fn}"


def test_host_side_validation(lib):
    out = ctypes.c_void_p()
    p = (ctypes.c_int32 * 1)(4)
    assert lib.mps_create_batch(0, p, None, 4, 1, None, ctypes.byref(out)) == 1
    assert b"n_images" in lib.mps_last_error()
    assert lib.mps_create_batch(1, None, None, 4, 1, None, ctypes.byref(out)) == 1
    assert lib.mps_create_batch(1, p, None, 4, 9, None, ctypes.byref(out)) == 1
    bad = (ctypes.c_int32 * 1)(17)
    assert lib.mps_create_batch(1, bad, None, 4, 1, None, ctypes.byref(out)) == 1
    assert lib.mps_create_batch(1, p, None, 0, 1, None, ctypes.byref(out)) == 1
    assert lib.mps_create_batch(1, p, None, 4097, 1, None, ctypes.byref(out)) == 1   # above MPS_CHI_LIMIT
    assert lib.mps_create_batch(1, p, None, 4, 1, None, None) == 1
    assert lib.mps_destroy_batch(None) == 0
    assert lib.mps_sync(None) == 1
    assert lib.ano_features(None, 0, 1, 1, None, None, None, 0, None, None, None) == 1
    # refused before any launch: the (host) buffers are never read
    buf = (ctypes.c_float * 16)()
    assert lib.ano_features(buf, 0, 1 << 31, 1, buf, None, None, 0, buf, None, None) == 1
    assert b"2^31" in lib.mps_last_error()


def test_pair_counts(lib):
    for p in range(2, 17):
        assert lib.mps_pair_count(p, 0) == 2 * p * (p - 1)
        assert lib.mps_pair_count(p, 1) == 2 * p * (p - 1) + 2 * (p - 1) ** 2
    assert lib.mps_pair_count(7, 1) == 156       # Sec. II.C
    assert isinstance(lib.mps_launch_count(), int)


def test_training_entry_validation(lib):
    """ano_train_step rejects bad arguments on the host, before any device work."""
    assert lib.ano_train_workspace_floats(0, 84, 784) == -1
    n = lib.ano_train_workspace_floats(1024, 84, 784)
    assert n >= 2 * 1024 * 84 + 1024 * 784 + 84 * 16 + 784 * 84 + 784
    hp = _lib.ano_adam(1e-2, 1e-3, 0.9, 0.999, 1e-8, 1.0)
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    args = [fake, 0, 8, 4, fake, fake, fake, 10, fake, fake, 1, ctypes.byref(hp), fake, fake, None]
    a = list(args); a[0] = None
    assert lib.ano_train_step(*a) == 1
    a = list(args); a[10] = 0                       # Adam steps count from 1
    assert lib.ano_train_step(*a) == 1 and b"step" in lib.mps_last_error()
    bad = _lib.ano_adam(1e-2, 1e-3, 1.0, 0.999, 1e-8, 1.0)
    a = list(args); a[11] = ctypes.byref(bad)
    assert lib.ano_train_step(*a) == 1
    a = list(args); a[12] = ctypes.c_void_p(0x1004)  # workspace not 8-byte aligned
    assert lib.ano_train_step(*a) == 1 and b"aligned" in lib.mps_last_error()
