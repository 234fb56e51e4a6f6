"""Out-of-memory paths through the library's allocation cap
(gx_set_device_memory_cap): a scene set, a context and a training run that do
not fit return GX_ENOMEM, release everything they had allocated (the bytes
the library holds come back to what they were), and the library works again
once the cap is lifted.  No device memory is exhausted for real."""
import numpy as np
import pytest

from paper_2306_07552_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
GX_ENOMEM = 2


def test_allocation_cap_gives_enomem_without_leaks():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scenes = I.make_scenes(I.WORKLOADS["apartments4096"], only=[0, 1])
    gx.set_device_memory_cap(0)
    u0 = gx.device_memory_in_use()
    cap = u0 + (8 << 20)
    try:
        gx.set_device_memory_cap(cap)
        # the dense grids (~100 MB each) do not fit: refused, nothing kept
        with pytest.raises(gx.GxError) as ei:
            gx.SceneSet(scenes)
        assert ei.value.status == GX_ENOMEM
        assert gx.device_memory_in_use() == u0
        # without dense grids the same scenes fit under the cap
        lean = gx.SceneSet(scenes, dense_grid=False, column_grid=False)
        u1 = gx.device_memory_in_use()
        assert u0 < u1 <= cap
        # a context whose framebuffer slots and state do not fit
        with pytest.raises(gx.GxError) as ei:
            gx.Sim(lean, ROBOT, 4096, img=(128, 128), n_objects=40, static_store=1)
        assert ei.value.status == GX_ENOMEM
        assert gx.device_memory_in_use() == u1
        # weights fit; the training set (16 bytes per sample) does not
        gx.set_device_memory_cap(u1 + (1 << 20))
        lean.nsdf_set_weights(0, I.fourier_matrix(7), I.nsdf_init(7))
        u2 = gx.device_memory_in_use()
        with pytest.raises(gx.GxError) as ei:
            lean.nsdf_train(0, n_samples=1_000_000, batch=65536, steps=10, lr=1e-3, seed=1)
        assert ei.value.status == GX_ENOMEM
        assert gx.device_memory_in_use() == u2
    finally:
        gx.set_device_memory_cap(0)
    # the cap lifted: the same calls succeed, and closing returns every byte
    sim = gx.Sim(lean, ROBOT, 64, img=(64, 64), n_objects=8, static_store=1)
    sim.reset()
    out = sim.step(torch.zeros((64, 11), device="cuda"))
    torch.cuda.synchronize()
    assert out["depth"].abs().sum().item() > 0
    assert sim.device_error() == 0
    losses = lean.nsdf_train(0, n_samples=200_000, batch=65536, steps=5, lr=1e-3, seed=1)
    assert np.all(np.isfinite(losses))
    sim.close()
    lean.close()
    assert gx.device_memory_in_use() == u0
