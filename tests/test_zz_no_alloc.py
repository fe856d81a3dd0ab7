"""mc_sweep_noalloc: FP32 sweeps for callers that cannot allocate device
memory (a framework's pool owns the GPU, or the surrounding loop forbids
cudaMalloc and the synchronisation it brings).  The entry point takes the
caller's device buffers and keeps its own scratch in a static device array.

Checked against the allocating path (mc_create_ex / mc_import_state /
mc_sweep): two calls in a row, each continuing the chain, give the same spins,
cone angle and per-sweep samples.  The module runs last (its name sorts
last), works in a fresh process as well as after the other tests, and needs
a GPU.
"""
import ctypes

import numpy as np
import pytest

import paper_2103_03517_gb300 as mc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


def _reference(dims, kw, n1, n2):
    """Two mc_sweep calls through the allocating path: initial raw state,
    spins and samples after each call, cone angles."""
    h = mc.mc_create_ex(mc.make_desc(dims, ring_capacity=n1 + n2, **kw))
    try:
        nbytes = mc.mc_state_bytes(h)
        start = np.zeros(nbytes // 4, np.float32)
        mc.mc_export_state(h, start.ctypes.data, nbytes)
        out = []
        for n in (n1, n2):
            mc.mc_sweep(h, n, measure=True)
            spins = np.zeros_like(start)
            mc.mc_export_state(h, spins.ctypes.data, nbytes)
            theta, _ = mc.mc_get_theta(h)
            out.append((spins, theta))
        samples = mc.mc_samples(h, n1 + n2)
    finally:
        mc.mc_destroy(h)
    return start, out, samples


# (16, 16, 16) and (64, 32, 8) take the row kernel; (12, 6, 4), with rows of
# 6 sites per colour, takes the general colour kernel
@pytest.mark.parametrize("dims", [(16, 16, 16), (64, 32, 8), (12, 6, 4)])
def test_noalloc_matches_allocating_path_on_two_calls(dims):
    torch = pytest.importorskip("torch")
    kw = dict(J=1.0, K_u=0.05, K_c=0.02, H=(0.0, 0.0, 0.1), T=0.8, seed=21)
    n1, n2 = 23, 17
    start, ref, ref_samples = _reference(dims, kw, n1, n2)

    spins = torch.from_numpy(start).cuda()             # caller-owned device memory
    samples = torch.zeros((n1 + n2) * 14, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    theta = 30
    first = 0
    for k, n in enumerate((n1, n2)):
        sp = samples.data_ptr() + (first * 14) * 8
        theta = mc.mc_sweep_noalloc(spins.data_ptr(), dims, kw["J"], kw["K_u"], (0.0, 0.0, 1.0), kw["K_c"],
                                    kw["H"], kw["T"], kw["seed"], first, n, theta, samples_ptr=sp)
        first += n
        got = spins.cpu().numpy()
        want, want_theta = ref[k]
        np.testing.assert_allclose(got, want, rtol=0, atol=0)   # same kernels: identical bits
        assert theta == want_theta
    s = samples.cpu().numpy().reshape(n1 + n2, 14)
    assert np.array_equal(s[:, 0].astype(np.int64), ref_samples["sweep"])
    assert np.array_equal(s[:, 1].astype(np.int32), ref_samples["theta_deg"])
    assert np.array_equal(s[:, 2].astype(np.int64), ref_samples["accepted"])
    np.testing.assert_allclose(s[:, 3:6], ref_samples["m"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(s[:, 6:10], ref_samples["e_parts"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(s[:, 10:13], ref_samples["torque"], rtol=0, atol=1e-12)


def test_noalloc_rejects_oversize_sample_request():
    torch = pytest.importorskip("torch")
    dims = (16, 16, 16)
    spins = torch.zeros(6 * 2048, dtype=torch.float32, device="cuda")
    samples = torch.zeros(300 * 14, dtype=torch.float64, device="cuda")
    with pytest.raises(mc.MCError) as e:
        mc.mc_sweep_noalloc(spins.data_ptr(), dims, 1.0, 0.0, (0, 0, 1.0), 0.0, (0, 0, 0), 1.0, 0, 0, 300, 30,
                            samples_ptr=samples.data_ptr())
    assert e.value.code == mc.MC_ERR_ARG and "256" in str(e.value)


def test_noalloc_call_leaves_free_device_memory_unchanged():
    """After a first call (which loads the kernels), further calls take no
    device memory: the free bytes the driver reports do not move."""
    torch = pytest.importorskip("torch")
    dims = (32, 32, 32)
    h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.01, T=0.9, seed=5))
    try:
        nbytes = mc.mc_state_bytes(h)
        start = np.zeros(nbytes // 4, np.float32)
        mc.mc_export_state(h, start.ctypes.data, nbytes)
    finally:
        mc.mc_destroy(h)
    spins = torch.from_numpy(start).cuda()
    samples = torch.zeros(16 * 14, dtype=torch.float64, device="cuda")
    args = (dims, 1.0, 0.01, (0.0, 0.0, 1.0), 0.0, (0.0, 0.0, 0.0), 0.9, 5)
    theta = mc.mc_sweep_noalloc(spins.data_ptr(), *args, 0, 8, 30, samples_ptr=samples.data_ptr())
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    first = 8
    for _ in range(3):
        theta = mc.mc_sweep_noalloc(spins.data_ptr(), *args, first, 16, theta, samples_ptr=samples.data_ptr())
        first += 16
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
