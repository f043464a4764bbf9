"""CPU checks of the C ABI library: it loads without a GPU, exports every entry
point include/vplbm.h declares, and its host-only helpers behave."""
import ctypes
import os
import re

import pytest

from paper_1812_05401_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(vplbm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1812_05401_gb300 import vplbm as V
    return V.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("vplbm_create", "vplbm_set_mask_and_solid_velocity", "vplbm_step",
                     "vplbm_moments", "vplbm_forces", "vplbm_destroy", "vplbm_group_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_helpers(lib):
    from paper_1812_05401_gb300 import vplbm as V
    assert V.vplbm_tau_from_reynolds(0.05, 40.0, 100.0) == pytest.approx(0.56)
    c = V.make_config(1024, 256, "mrt", "f32")
    fp = V.vplbm_footprint_bytes(c)
    # two population buffers of 9 x 1024 x 256 FP32 dominate
    assert 2 * 9 * 1024 * 256 * 4 < fp < 2 * 9 * 1024 * 256 * 4 * 1.05
    c16 = V.make_config(1024, 256, "mrt", "f16")
    assert V.vplbm_footprint_bytes(c16) < 0.55 * fp
    bad = V.make_config(0, 10)
    assert V.vplbm_footprint_bytes(bad) == 0
    # in-place streaming keeps one population buffer (plus 9 values per row
    # of side state at open x sides)
    ab = V.make_config(16384, 4096, "mrt", "f32", 0.6, bc="channel")
    aa = V.make_config(16384, 4096, "mrt", "f32", 0.6, bc="channel", streaming="aa")
    fab, faa = V.vplbm_footprint_bytes(ab), V.vplbm_footprint_bytes(aa)
    assert fab - faa == 9 * 16384 * 4096 * 4 - 9 * 4096 * 4
    assert faa < 0.55 * fab
    assert V.lib().vplbm_status_string(4) == b"diverged"


def test_invalid_configs_rejected_without_gpu(lib):
    from paper_1812_05401_gb300 import vplbm as V
    for kw in (dict(nx=0, ny=4), dict(nx=4, ny=4, tau=0.5), dict(nx=4, ny=4, eta=0.0),
               dict(nx=4, ny=4, storage=7), dict(nx=4, ny=4, ring_len=0),
               dict(nx=4, ny=4, streaming=2), dict(nx=4, ny=4, bc=(3, 2), u_in=(0.05, 0.0),
                                                   u_conv=-1.0),
               dict(nx=1 << 17, ny=1 << 18),  # 2^35 nodes: beyond the 2^34 limit
               dict(nx=4, ny=4, rounding=5), dict(nx=4, ny=4, collision=2),
               dict(nx=4, ny=4, bc=(2, 0)),  # free slip is a y condition only
               dict(nx=4, ny=4, bc=(0, 1)),  # inlet/outlet is an x condition only
               dict(nx=4, ny=4, tau=float("nan")), dict(nx=4, ny=4, rho0=0.0),
               dict(nx=4, ny=4, collision="mrt", lam=0.0)):
        nx, ny = kw.pop("nx"), kw.pop("ny")
        c = V.make_config(nx, ny, **kw)
        with pytest.raises(V.VplbmError) as e:
            V.vplbm_create(c)
        assert e.value.status == V.VPLBM_ERR_INVALID
        # the reason travels with the error (no handle exists to carry it)
        why = V.lib().vplbm_create_error().decode()
        assert why and why in str(e.value)
    c = V.make_config(4, 4, tau=0.5)
    with pytest.raises(V.VplbmError, match="tau must be > 1/2"):
        V.vplbm_create(c)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1812_05401_gb300 import vplbm as V
    monkeypatch.setattr(V, "_lib", None)
    monkeypatch.setattr(V, "LIB_PATH", str(tmp_path / "libvplbm.so"))
    with pytest.raises(ImportError):
        V.lib()


def test_header_and_library_from_c(lib, tmp_path):
    """The header is plain C: a C program compiled against it and linked with
    libvplbm.so makes the host-only calls (no GPU needed)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1812_05401_gb300")
    exe = str(tmp_path / "abi_host_calls")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                    os.path.join(root, "tests", "c", "abi_host_calls.c"), "-o", exe,
                    "-L", pkg, "-lvplbm", "-Wl,-rpath," + pkg, "-lm"], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_binding_structs_match_the_header(tmp_path):
    """Every field of the ctypes vplbm_config and vplbm_body sits at the
    offset and has the size a C compiler gives it from the header (the
    binding's `lam` is the header's `lambda`)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_1812_05401_gb300 import vplbm as V
    exe = str(tmp_path / "abi_layout")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_layout.c"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60, check=True).stdout
    structs = {"vplbm_config": V.vplbm_config, "vplbm_body": V.vplbm_body}
    rename = {"lambda": "lam"}
    seen = {name: [] for name in structs}
    for line in out.split("\n"):
        if not line:
            continue
        sname, field, *nums = line.split()
        S = structs[sname]
        if field == "sizeof":
            assert ctypes.sizeof(S) == int(nums[0]), (sname, ctypes.sizeof(S), nums)
            continue
        desc = getattr(S, rename.get(field, field))
        assert (desc.offset, desc.size) == (int(nums[0]), int(nums[1])), (sname, field, nums)
        seen[sname].append(rename.get(field, field))
    for sname, S in structs.items():
        assert seen[sname] == [f[0] for f in S._fields_], sname


def test_torch_allocator_binds_one_stream_without_gpu():
    """The binding's stream rule for the device memory hook, on raw handles
    (no CUDA call): the allocator's stream becomes the config's; a config on
    another stream, or the legacy NULL stream, is refused."""
    from paper_1812_05401_gb300 import vplbm as V
    A = V.TorchAllocator(stream=0x1230, device=0)
    c = V.make_config(64, 32, allocator=A)
    assert c.stream == 0x1230 and bool(c.dev_alloc) and bool(c.dev_free)
    assert c._allocator is A and A.allocs == A.frees == 0
    assert V.make_config(64, 32, stream=0x1230, allocator=A).stream == 0x1230
    with pytest.raises(ValueError):
        V.make_config(64, 32, stream=0x4560, allocator=A)
    with pytest.raises(ValueError):
        V.make_config(64, 32, allocator=V.TorchAllocator(stream=0, device=0))
    # a config's own stream binds an allocator made without one
    B = V.TorchAllocator(device=0)
    assert V.make_config(64, 32, stream=0x7890, allocator=B).stream == 0x7890
    assert B.stream == 0x7890


def test_c_example_builds_against_the_header(lib, tmp_path):
    """tests/c/example_cylinder.c, the C usage example, compiles and links
    with -Wall -Werror (running it needs a GPU)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    pkg = os.path.join(ROOT, "paper_1812_05401_gb300")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "example_cylinder.c"), "-o",
                    str(tmp_path / "cylinder"), "-L", pkg, "-lvplbm", "-Wl,-rpath," + pkg],
                   check=True)
    assert os.path.exists(tmp_path / "cylinder")
