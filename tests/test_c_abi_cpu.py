"""The C ABI from a plain C program (no GPU work): include/dmcr.h compiles as C, libdmcr
links into a C client, the host-side calls answer as documented, and the ctypes structs of
the Python binding have exactly the C layout."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2103_09686_gb300 import _build, _lib
    _lib.load(build_if_missing=True)
    libdir = os.path.dirname(_build.LIB)
    exe = str(tmp_path_factory.mktemp("cabi") / "probe")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_probe.c"), "-o", exe, "-L", libdir, "-ldmcr",
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    sizes, offsets, values = {}, {}, {}
    for line in out.splitlines():
        kind, name, *rest = line.split()
        if kind == "size":
            sizes[name] = int(rest[0])
        elif kind == "offset":
            offsets[name] = int(rest[0])
        else:
            values[kind] = [int(x) for x in [name] + rest]
    return sizes, offsets, values


@pytest.mark.parametrize("name", ["dmcr_params", "dmcr_loss_opts", "dmcr_recon_opts", "dmcr_adam_state",
                                  "dmcr_recon_report"])
def test_binding_structs_have_the_c_layout(probe, name):
    from paper_2103_09686_gb300 import _lib
    sizes, offsets, _ = probe
    cls = getattr(_lib, name)
    assert ctypes.sizeof(cls) == sizes[name]
    fields = [f[0] for f in cls._fields_]
    assert sorted(fields) == sorted(k.split(".", 1)[1] for k in offsets if k.startswith(name + "."))
    for f in fields:
        assert getattr(cls, f).offset == offsets[name + "." + f], f


def test_host_calls_from_c(probe):
    from paper_2103_09686_gb300 import _lib
    _, _, v = probe
    assert v["version"][0] >= 100
    assert v["length_64_16"] == [_lib.DMCR_OK, 545]
    assert v["length_512_64_3"] == [_lib.DMCR_OK, 3 * 8321]
    assert v["workspace_512_64_3"][0] == _lib.DMCR_OK and v["workspace_512_64_3"][1] > 0
    assert v["invalid"] == [_lib.DMCR_EINVAL, 1]
    assert v["null_params"] == [_lib.DMCR_EINVAL]
    assert v["null_workspace"] == [_lib.DMCR_EINVAL]
