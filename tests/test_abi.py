"""The C-ABI library builds, loads and exports every entry point the header declares.

These run without a GPU: only symbol lookup and argument checks that return
before any CUDA call.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(onng_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1810_07355_gb300 import onng
    return onng.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 16
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1810_07355_gb300 import onng
    assert set(onng.exported_symbols()) <= _declared()


def test_version_and_argument_checks(lib):
    from paper_1810_07355_gb300 import onng
    assert lib.onng_version() >= 1
    # rejected before any CUDA call: bad sizes, unsupported d / k
    st = lib.onng_knn(None, 10, 6, None, 10, 5, -1, None, None, None, 0, None)
    assert st == onng.ONNG_E_UNSUPPORTED and b"multiple of 4" in lib.onng_last_error()
    st = lib.onng_knn(None, 10, 8, None, 10, 500, -1, None, None, None, 0, None)
    assert st == onng.ONNG_E_UNSUPPORTED
    st = lib.onng_knn(None, -1, 8, None, 10, 5, -1, None, None, None, 0, None)
    assert st == onng.ONNG_E_INVAL
    st = lib.onng_seeds_random(1, 4, 100, 0, None, None)
    assert st == onng.ONNG_E_UNSUPPORTED
    st = lib.onng_seeds_random(1, 4, 0, 4, None, None)
    assert st == onng.ONNG_E_INVAL
    p = onng._Params(0, 10, 0.1, 0, 0, 0)
    ix = onng._Index(None, None, None, None, None, 100, 128, 0)
    st = lib.onng_search(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None, 0, None)
    assert st == onng.ONNG_E_UNSUPPORTED and b"k must be" in lib.onng_last_error()
    ix = onng._Index(None, None, None, None, None, 100, 130, 0)
    p = onng._Params(10, 10, 0.1, 0, 0, 0)
    st = lib.onng_search(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None, 0, None)
    assert st == onng.ONNG_E_UNSUPPORTED
    st = lib.onng_adjust_degree_count(None, None, -5, 10, 3, 3, None, None, None, 0, None)
    assert st == onng.ONNG_E_INVAL
    ix = onng._Index(None, None, None, None, None, 100, 128, 0)
    p = onng._Params(10, 10, 0.1, 0, 0, 0, -1)
    st = lib.onng_search(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None, 0, None)
    assert st == onng.ONNG_E_INVAL and b"pool_cap" in lib.onng_last_error()


def test_reduced_precision_argument_checks(lib):
    """Rejected before any CUDA call: FP8 search without its codes or scales, a
    bf16 search without X_bf16, bad FP8 conversion arguments, unknown precision."""
    from paper_1810_07355_gb300 import onng
    ix = onng._Index(None, None, None, None, None, 100, 128, 0)
    p = onng._Params(10, 10, 0.1, onng.PREC_FP8, 20, 0)
    st = lib.onng_search(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None, 0, None)
    assert st == onng.ONNG_E_INVAL and b"fp8 needs" in lib.onng_last_error()
    p = onng._Params(10, 10, 0.1, onng.PREC_BF16, 20, 0)
    st = lib.onng_search(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None, 0, None)
    assert st == onng.ONNG_E_INVAL and b"bf16 needs" in lib.onng_last_error()
    p = onng._Params(10, 10, 0.1, 7, 20, 0)
    st = lib.onng_search(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None, 0, None)
    assert st == onng.ONNG_E_INVAL and b"unknown precision" in lib.onng_last_error()
    p = onng._Params(10, 10, 0.1, onng.PREC_FP8, 200, 0)
    st = lib.onng_search(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None, 0, None)
    assert st == onng.ONNG_E_UNSUPPORTED and b"k_rerank" in lib.onng_last_error()
    assert lib.onng_to_fp8(None, -1, 8, None, None, None) == onng.ONNG_E_INVAL
    assert lib.onng_to_fp8(None, 10, 8, None, None, None) == onng.ONNG_E_INVAL


def test_crc32_matches_zlib(lib):
    import zlib
    from paper_1810_07355_gb300 import onng
    rng = os.urandom(4099)
    for data in (b"", b"123456789", rng):
        assert onng.crc32(data) == zlib.crc32(data)
    # continuation: the CRC of a + b from the CRC of a
    assert onng.crc32(rng[1000:], onng.crc32(rng[:1000])) == zlib.crc32(rng)
    assert onng.crc32(b"123456789") == 0xCBF43926  # the published check value


def _write_index_file(path, row_ptr, col, length, X, version=1, crc=None):
    """An index file written from the layout the header documents."""
    import struct
    import zlib
    payload = row_ptr.astype("<i8").tobytes() + col.astype("<i4").tobytes()
    if length is not None:
        payload += length.astype("<f4").tobytes()
    payload += X.astype("<f4").tobytes()
    c = zlib.crc32(payload) if crc is None else crc
    head = b"ONNGIDX\0" + struct.pack("<IIqiIq", version, 1 if length is not None else 0, len(row_ptr) - 1,
                                      X.shape[1], c, len(col)) + bytes(24)
    assert len(head) == 64
    with open(path, "wb") as f:
        f.write(head + payload)


def test_index_file_check(lib, tmp_path):
    import numpy as np
    from paper_1810_07355_gb300 import onng
    rng = np.random.default_rng(0)
    rp = np.array([0, 2, 3, 5], np.int64)
    col = np.array([1, 2, 0, 0, 1], np.int32)
    ln = rng.random(5).astype(np.float32)
    X = rng.random((3, 8)).astype(np.float32)
    good = tmp_path / "g.onng"
    _write_index_file(good, rp, col, ln, X)
    assert onng.index_check(str(good)) == {"n": 3, "d": 8, "nnz": 5, "has_len": True}
    _write_index_file(good, rp, col, None, X)
    assert onng.index_check(str(good))["has_len"] is False
    bad = tmp_path / "b.onng"
    for kw, msg in ((dict(version=2), b"version"), (dict(crc=1), b"CRC")):
        _write_index_file(bad, rp, col, ln, X, **kw)
        with pytest.raises(onng.OnngError):
            onng.index_check(str(bad))
        assert msg in lib.onng_last_error()
    # one flipped payload byte, a truncated file, a missing file
    _write_index_file(bad, rp, col, ln, X)
    raw = bytearray(bad.read_bytes())
    raw[100] ^= 1
    bad.write_bytes(bytes(raw))
    with pytest.raises(onng.OnngError):
        onng.index_check(str(bad))
    bad.write_bytes(bytes(raw[:-4]))
    with pytest.raises(onng.OnngError):
        onng.index_check(str(bad))
    with pytest.raises(onng.OnngError):
        onng.index_check(str(tmp_path / "missing.onng"))
    # a load whose sizes disagree with the file is refused before any CUDA call
    _write_index_file(good, rp, col, ln, X)
    st = lib.onng_index_load(str(good).encode(), 4, 8, 5, C.c_void_p(8), C.c_void_p(8), None, C.c_void_p(8), None)
    assert st == onng.ONNG_E_INVAL and b"expects" in lib.onng_last_error()


def test_serve_argument_checks(lib):
    from paper_1810_07355_gb300 import onng
    out = C.c_void_p()
    cfg = onng._ServeConfig(0, 0, 256, 10, 64, 10, 2, 1000)
    st = lib.onng_serve_create(None, C.byref(cfg), C.byref(out))
    assert st == onng.ONNG_E_INVAL and out.value is None
    ix = onng._Index(None, None, C.c_void_p(16), None, None, 100, 128, 0)
    for bad in (onng._ServeConfig(0, 0, 256, 10, 64, 10, 0, 1000), onng._ServeConfig(0, 0, 256, 10, 0, 10, 2, 1000),
                onng._ServeConfig(0, 0, 256, 10, 64, 10, 2, 0)):
        assert lib.onng_serve_create(C.byref(ix), C.byref(bad), C.byref(out)) == onng.ONNG_E_INVAL
    assert lib.onng_serve_destroy(None) == onng.ONNG_OK


def test_header_is_plain_c_and_a_c_program_links(lib, tmp_path):
    """include/onng.h compiles as C99 (warnings as errors, -pedantic) and a C
    program linked against libonng.so calls it with no Python in the process: the
    version, the index-file CRC-32 (check value 0xCBF43926 on "123456789") and an
    argument error reported through onng_last_error before any device work."""
    import shutil
    import subprocess
    from paper_1810_07355_gb300 import build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "onng.h"

int main(void)
{
    int st;
    if (onng_version() < 1)
        return 1;
    if (onng_crc32(0u, "123456789", 9) != 0xCBF43926u)
        return 2;
    st = onng_knn(NULL, 10, 6, NULL, 10, 5, -1, NULL, NULL, NULL, 0, NULL);
    if (st != ONNG_E_UNSUPPORTED || strstr(onng_last_error(), "multiple of 4") == NULL)
        return 3;
    st = onng_seeds_random(1u, 4, 0, 4, NULL, NULL);
    if (st != ONNG_E_INVAL)
        return 4;
    printf("c abi ok %d\n", onng_version());
    return 0;
}
""")
    libdir = os.path.dirname(build.LIB)
    exe = str(tmp_path / "abi")
    cmd = [gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", exe, "-L", libdir, "-lonng", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.startswith("c abi ok"), (r.returncode, r.stdout, r.stderr)


def test_status_codes_match_header():
    """The binding's status constants are the header's enum values."""
    from paper_1810_07355_gb300 import onng
    text = open(os.path.join(ROOT, "include", "onng.h")).read()
    body = re.search(r"enum onng_status \{(.*?)\};", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    enum = {m.group(1): int(m.group(2)) for m in re.finditer(r"(ONNG_\w+)\s*=\s*(\d+)", body)}
    assert len(enum) == 7
    for name, value in enum.items():
        assert getattr(onng, name) == value, name


def test_last_error_is_per_thread(lib):
    """onng_last_error() is thread-local: two threads that fail differently each
    read back their own message after both have failed."""
    import threading
    from paper_1810_07355_gb300 import onng
    barrier = threading.Barrier(2)
    seen = {}

    def knn_fails():
        st = lib.onng_knn(None, 10, 6, None, 10, 5, -1, None, None, None, 0, None)
        barrier.wait()
        seen["knn"] = (st, lib.onng_last_error())

    def seeds_fail():
        st = lib.onng_seeds_random(1, 4, 100, 0, None, None)
        barrier.wait()
        seen["seeds"] = (st, lib.onng_last_error())

    threads = [threading.Thread(target=knn_fails), threading.Thread(target=seeds_fail)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert seen["knn"][0] == onng.ONNG_E_UNSUPPORTED and b"multiple of 4" in seen["knn"][1]
    assert seen["seeds"][0] == onng.ONNG_E_UNSUPPORTED and b"n_seed" in seen["seeds"][1]
    assert b"n_seed" not in seen["knn"][1] and b"multiple of 4" not in seen["seeds"][1]


def test_missing_library_fails_loudly(tmp_path):
    """With the library missing the binding raises on first use; nothing falls
    back to another implementation (checked in a child process, so this one keeps
    its loaded library)."""
    import subprocess
    import sys
    child = (
        "from paper_1810_07355_gb300 import onng\n"
        "for call in (onng.load, lambda: onng.crc32(b'123456789')):\n"
        "    try:\n"
        "        call()\n"
        "    except RuntimeError as e:\n"
        "        assert 'not found' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('no error')\n"
        "print('raised')\n")
    env = dict(os.environ, ONNG_LIBRARY=str(tmp_path / "missing" / "libonng.so"), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", child], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "raised" in r.stdout, r.stdout + r.stderr
