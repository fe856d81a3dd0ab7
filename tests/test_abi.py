"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/mc.h, its structs have the layout the binding assumes,
and host-side argument checks reject invalid descriptions before any CUDA
call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2103_03517_gb300 as mc
from paper_2103_03517_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mc.h")


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"MC_API\s+[\w\s\*]+?\b(mc_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("mc_create", "mc_create_ex", "mc_sweep", "mc_constrained_sweep", "mc_measure",
                 "mc_submit", "mc_poll", "mc_group_sweep", "mc_save", "mc_load"):
        assert name in syms
    assert len(syms) >= 30


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(libbuild.LIB)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(declared_symbols()), exported ^ set(declared_symbols())


def test_binding_covers_every_symbol():
    for name in declared_symbols():
        assert name in mc._mc._SIGS, name


def test_struct_layout_matches_c():
    src = os.path.join(ROOT, "_build", "sizes.c")
    exe = os.path.join(ROOT, "_build", "sizes")
    os.makedirs(os.path.dirname(src), exist_ok=True)
    with open(src, "w") as f:
        f.write('#include "mc.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                'sizeof(mc_desc),sizeof(mc_observables),sizeof(mc_sample),sizeof(mc_job),sizeof(mc_result),'
                'sizeof(mc_server_desc),offsetof(mc_desc,stream),offsetof(mc_observables,binder));return 0;}\n')
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
    got = list(map(int, subprocess.run([exe], capture_output=True, text=True).stdout.split()))
    want = [ctypes.sizeof(mc.mc_desc), ctypes.sizeof(mc.mc_observables), ctypes.sizeof(mc.mc_sample),
            ctypes.sizeof(mc.mc_job), ctypes.sizeof(mc.mc_result), ctypes.sizeof(mc.mc_server_desc),
            mc.mc_desc.stream.offset, mc.mc_observables.binder.offset]
    assert got == want


def test_desc_defaults():
    d = mc.mc_desc_default()
    assert list(d.dims) == [16, 16, 16] and d.precision == mc.MC_FP32 and d.theta0_deg == 30
    assert d.J == 1.0 and list(d.axis) == [0, 0, 1.0] and d.ring_capacity == 4096


@pytest.mark.parametrize("kw,msg", [
    (dict(dims=(15, 16, 16), boundary=(1, 0, 0)), "even"),
    (dict(dims=(15, 16, 16)), "odd size"),
    (dict(dims=(16, 15, 16)), "odd size"),
    (dict(dims=(16, 16, 15), boundary=(0, 0, 3)), "odd size"),
    (dict(dims=(16, 16, 16), T=0.0), "T must"),
    (dict(dims=(16, 16, 16), T=-1.0), "T must"),
    (dict(dims=(16, 16, 16), axis=(0, 0, 0)), "axis"),
    (dict(dims=(16, 16, 16), theta0_deg=0), "theta0"),
    (dict(dims=(16, 16, 16), theta0_deg=181), "theta0"),
    (dict(dims=(0, 16, 16)), "dims"),
    (dict(dims=(2048, 2048, 1024)), "2^32"),
    (dict(dims=(16, 16, 16), precision=7), "precision"),
    (dict(dims=(16, 16, 16), boundary=(0, 0, 5)), "boundary"),
])
def test_invalid_descriptions_rejected_on_host(kw, msg):
    d = mc.make_desc(**kw)
    with pytest.raises(mc.MCError) as e:
        mc.mc_create_ex(d)
    assert e.value.code == mc.MC_ERR_ARG and msg in str(e.value)


def test_asymmetric_bond_mask_rejected():
    dims = (4, 4, 2)
    mask = np.full(32, 0x3F, np.uint8)
    mask[5] &= ~np.uint8(2)  # drop +x of site 5 only
    d = mc.make_desc(dims, boundary=(0, 0, 1), bond_mask=mask)
    with pytest.raises(mc.MCError) as e:
        mc.mc_create_ex(d)
    assert e.value.code == mc.MC_ERR_ARG and "symmetric" in str(e.value)


def test_grain_ids_out_of_range_rejected():
    d = mc.make_desc((4, 4, 2), boundary=(0, 0, 1), grain_id=np.full(32, 3, np.int32),
                     grain_axis=np.eye(3))
    with pytest.raises(mc.MCError) as e:
        mc.mc_create_ex(d)
    assert e.value.code == mc.MC_ERR_ARG


def test_null_handles_rejected():
    with pytest.raises(mc.MCError):
        mc.mc_sweep(None, 1)
    with pytest.raises(mc.MCError):
        mc.mc_measure(None)
    with pytest.raises(mc.MCError) as e:
        mc.mc_group_measure(None, 4)
    assert e.value.code == mc.MC_ERR_ARG
    assert mc.mc_destroy(None) is None


def test_noalloc_object_calls_no_allocation_routine():
    """The object of mc_sweep_noalloc references no allocating CUDA routine
    (device, host or stream-ordered memory, streams, events, graphs); the GPU
    test checks the free device memory across calls."""
    obj = os.path.join(ROOT, "_build", "libmc", "noalloc.cu.o")
    out = subprocess.run(["nm", "-u", obj], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    undefined = [ln.split()[-1] for ln in out.stdout.splitlines() if ln.strip()]
    assert any("cudaGetSymbolAddress" in u for u in undefined)
    banned = re.compile(r"cuda(Malloc|Free|HostAlloc|HostRegister|StreamCreate|EventCreate|Graph|MemPool)|cuMem")
    assert not [u for u in undefined if banned.search(u)]
