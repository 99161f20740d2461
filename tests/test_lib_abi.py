"""CPU-only checks of the C ABI library: it builds, loads, exports every symbol include/vbh.h
declares, validates configurations without touching a GPU, and its host-side bucket function
matches the paper's spatial hash (Sec. 5) with the primes from tests/golden/k1_spatial_hash.txt."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    from paper_1805_03709_b300 import build
    build.build()
    from paper_1805_03709_b300 import vbh
    vbh.lib()
    return vbh


def read(*parts):
    with open(os.path.join(ROOT, *parts), encoding="utf-8") as f:
        return f.read()


def declared_functions():
    src = read("include", "vbh.h")
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vbh_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(V):
    names = declared_functions()
    assert len(names) >= 15
    bound = {s[0] for s in V.SYMBOLS}
    for n in names:
        assert hasattr(V.lib(), n), n
        assert n in bound, n


def test_abi_version(V):
    src = read("include", "vbh.h")
    ver = int(re.search(r"#define VBH_ABI_VERSION (\d+)", src).group(1))
    assert V.vbh_abi_version() == ver


def test_paper_spatial_hash(V):
    primes = {}
    for line in read("tests", "golden", "k1_spatial_hash.txt").splitlines():
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            primes[k] = int(v)
    rng = np.random.default_rng(0)
    for n_buckets in (2, 1 << 10, 1 << 22):
        for x, y, z in rng.integers(-(1 << 20), 1 << 20, size=(200, 3)).tolist() + [[0, 0, 0], [-1, -1, -1]]:
            m = 0xFFFFFFFF
            b = ((x * primes["p1"]) & m) ^ ((y * primes["p2"]) & m) ^ ((z * primes["p3"]) & m)
            assert V.vbh_bucket_of(x, y, z, n_buckets, V.VBH_HASH_PRIMES) == b % n_buckets
            assert V.vbh_bucket_of(x, y, z, n_buckets, V.VBH_HASH_MIX) < n_buckets
    assert V.vbh_bucket_of(1 << 20, 0, 0, 1024, 0) == V.VBH_NONE
    assert V.vbh_bucket_of(0, 0, 0, 1000, 0) == V.VBH_NONE


def test_mix_hash_spreads_a_contiguous_cube(V):
    n = 1 << 12
    counts = np.zeros(n, np.int64)
    for x in range(16):
        for y in range(16):
            for z in range(16):
                counts[V.vbh_bucket_of(x, y, z, n, V.VBH_HASH_MIX)] += 1
    assert counts.max() <= 8   # 4096 keys over 4096 buckets


@pytest.mark.parametrize("field,value", [("n_buckets", 1000), ("n_buckets", 0),
                                         ("slots_per_bucket", 8), ("hash_fn", 5),
                                         ("voxel_size", 0.0), ("width", 0), ("trunc", -1.0)])
def test_create_rejects_bad_config_before_any_device_work(V, field, value):
    cfg = V.vbh_config(voxel_size=0.01, trunc=0.04, max_weight=64, depth_scale=0.001, zmax=0,
                       width=8, height=8, fx=4, fy=4, cx=4, cy=4, n_buckets=1024,
                       slots_per_bucket=4, max_blocks=16, hash_fn=1, max_batch=0)
    setattr(cfg, field, value)
    with pytest.raises(V.VbhError) as e:
        V.vbh_create(cfg, None)
    assert e.value.status == V.VBH_ERR_INVALID_ARG


def test_struct_layouts_match_the_header(V, tmp_path):
    """Size and field offsets of every ctypes mirror equal the C compiler's for vbh.h."""
    import ctypes
    import subprocess
    names = [n for n in dir(V) if n.startswith("vbh_") and isinstance(getattr(V, n), type)
             and issubclass(getattr(V, n), ctypes.Structure)]
    assert len(names) >= 10
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vbh.h"', "int main(void) {"]
    for n in names:
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in getattr(V, n)._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for n in names:
        cls = getattr(V, n)
        assert int(got[n]) == ctypes.sizeof(cls), n
        for f, _ in cls._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(cls, f).offset, f"{n}.{f}"


def test_static_mc_entry_checks_its_arguments_before_any_device_work(V):
    """vbh_mc_from_tsdf_static refuses sizes beyond its fixed scratch and incomplete arguments
    with VBH_ERR_INVALID_ARG and a message, before it makes any CUDA call (so on the CPU too).
    The pointers below are never dereferenced."""
    import ctypes
    lib = V.lib()
    dummy = ctypes.c_uint32(0)
    addr = ctypes.addressof(dummy)
    out = V.vbh_mc_stream(addr, addr, addr, addr, addr, addr, 4, 4, addr, addr)
    cases = [(addr, (1 << 15) + 1, ctypes.byref(out), "32768"),
             (addr, 4, None, "null output"),
             (None, 4, ctypes.byref(out), "null input")]
    for keys, n, o, words in cases:
        st = lib.vbh_mc_from_tsdf_static(keys, keys, keys, n, o, None, None)
        assert st == V.VBH_ERR_INVALID_ARG
        assert words in lib.vbh_last_error().decode()
    incomplete = V.vbh_mc_stream(None, addr, addr, addr, addr, addr, 4, 4, addr, addr)
    st = lib.vbh_mc_from_tsdf_static(addr, addr, addr, 4, ctypes.byref(incomplete), None, None)
    assert st == V.VBH_ERR_INVALID_ARG
    assert "incomplete output" in lib.vbh_last_error().decode()


def test_diff_create_validates_its_config_before_any_device_work(V):
    """vbh_diff_create checks its configuration (and pointers) before any CUDA call: a bad one
    returns VBH_ERR_INVALID_ARG, names the rule in the last-error message and leaves *out null."""
    import ctypes
    lib = V.lib()
    good = dict(voxel_size=0.005, trunc=0.02, fx=262.5, fy=262.5, cx=160.0, cy=120.0, width=320,
                height=240, n_frames=64)
    for field, value in [("n_frames", 0), ("n_frames", 257), ("width", 1), ("trunc", 0.0),
                         ("voxel_size", float("nan")), ("fy", -1.0)]:
        cfg = V.vbh_diff_config(**dict(good, **{field: value}))
        out = ctypes.c_void_p(12345)
        st = lib.vbh_diff_create(ctypes.byref(cfg), None, ctypes.byref(out))
        assert st == V.VBH_ERR_INVALID_ARG, field
        assert out.value is None, field
        assert "n_frames in [1, 256]" in lib.vbh_last_error().decode()
    st = lib.vbh_diff_create(None, None, None)
    assert st == V.VBH_ERR_INVALID_ARG
    assert "null argument" in lib.vbh_last_error().decode()


def test_hash_batch_binding_refuses_wrong_arrays_before_the_library():
    """HashMap.batch checks shapes, dtypes and placement of its arrays in Python, before any
    library call (a wrong dtype would make the kernels read the bytes as something else)."""
    import torch
    from paper_1805_03709_b300.volume import HashMap
    hm = HashMap.__new__(HashMap)   # no device handle: every case below is refused first
    ops = torch.zeros(4, dtype=torch.uint8)
    keys = torch.zeros((4, 3), dtype=torch.int32)
    cases = [(ops, torch.zeros((5, 3), dtype=torch.int32), "keys3 [4, 3]"),
             (ops.to(torch.int32), keys, "ops must be torch.uint8"),
             (ops, keys.to(torch.int64), "keys3 must be torch.int32"),
             (ops, keys, "contiguous CUDA tensor")]
    for o, k, words in cases:
        with pytest.raises(ValueError, match=re.escape(words)):
            hm.batch(o, k)


def test_volume_key_lists_are_checked_before_the_library():
    """Volume.erase_keys and Volume.extract(keys3=...) pass block keys by pointer: anything but a
    dense [n, 3] int32 CUDA tensor is refused in Python."""
    import torch
    from paper_1805_03709_b300 import vbh as Vb
    from paper_1805_03709_b300.volume import Volume
    vol = Volume.__new__(Volume)   # no device handle: every case below is refused first
    for k, words in [(torch.zeros((4, 3), dtype=torch.int64), "int32 [n, 3]"),
                     (torch.zeros((4, 2), dtype=torch.int32), "int32 [n, 3]"),
                     (torch.zeros((4, 3), dtype=torch.int32), "contiguous CUDA tensor")]:
        with pytest.raises(ValueError, match=re.escape(words)):
            vol.erase_keys(k)
        with pytest.raises(ValueError, match=re.escape(words)):
            vol.extract(Vb.VBH_MC_KEYS, keys3=k, stream=object())


def test_static_mc_binding_refuses_wrong_arrays_before_the_library():
    """vbh.vbh_mc_from_tsdf_static checks dtypes, sizes and placement in Python before the
    library call: its kernels read 3 n int32 keys and 512 n floats from tsdf and weight and write
    one uint32 flag word, so any other layout would read or write out of bounds."""
    import torch
    from paper_1805_03709_b300 import vbh as Vb
    n = 4
    keys = torch.zeros((n, 3), dtype=torch.int32)
    F = torch.zeros((n, 512), dtype=torch.float32)
    err = torch.zeros(1, dtype=torch.int32)
    cases = [((keys.to(torch.int64), F, F, None), "keys3 must be int32 [n, 3]"),
             ((keys[:, :2], F, F, None), "keys3 must be int32 [n, 3]"),
             ((keys, F[:, :256], F, None), "tsdf must be float32 with n * 512"),
             ((keys, F, F.to(torch.float16), None), "weight must be float32 with n * 512"),
             ((keys, F.to(torch.float64), F, None), "tsdf must be float32"),
             ((keys, F, F, torch.zeros(1, dtype=torch.uint8)), "error_flags must be int32"),
             ((keys, F, F, torch.zeros(0, dtype=torch.int32)), "error_flags must be int32"),
             ((keys, F, F, err), "contiguous CUDA tensors"),
             ((keys, F.t(), F, None), "contiguous CUDA tensors")]
    for (k, t, w, e), words in cases:
        with pytest.raises(ValueError, match=re.escape(words)):
            Vb.vbh_mc_from_tsdf_static(k, t, w, None, None, e)
    # a host (numpy) array is refused as well
    with pytest.raises((ValueError, AttributeError)):
        Vb.vbh_mc_from_tsdf_static(keys.numpy(), F, F, None, None)
