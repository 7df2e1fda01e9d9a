"""Helpers for the GPU tests: raw-device-pointer views and store readback."""
import numpy as np


def device_view(addr, shape, typestr):
    """torch tensor aliasing device memory at a raw address (no copy)."""
    import torch

    class _A:
        pass
    a = _A()
    a.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(addr), False),
                                  "version": 3}
    return torch.as_tensor(a, device="cuda")


def read_store(cube, ctx):
    """The context's current store as numpy arrays (synchronises)."""
    import torch
    st = cube.cube_state_view(ctx)
    n, ncc = st.n_particles, st.n_coarse ** 3
    ct = "|i1" if st.x_bytes == 1 else "<i2"
    vt = "|i1" if st.v_bytes == 1 else "<i2"
    out = dict(
        counts=device_view(st.counts, (ncc,), "<u4").cpu().numpy().astype(np.int64),
        offsets=device_view(st.offsets, (ncc + 1,), "<u4").cpu().numpy().astype(np.int64),
        vc=device_view(st.vc, (3, ncc), "<f4").cpu().numpy(),
        chi=device_view(st.chi, (3, n), ct).cpu().numpy().astype(np.int64),
        nu=device_view(st.nu, (3, n), vt).cpu().numpy().astype(np.int64),
        ids=(device_view(st.id, (n,), {1: "|u1", 2: "<u2", 4: "<u4"}[st.id_bytes]).cpu().numpy().astype(np.uint32)
             if st.id else None),
        sigma=st.sigma, a=st.a, a_p=st.a_p, brick=st.brick, n_coarse=st.n_coarse)
    torch.cuda.synchronize()
    return out


def oracle_params(pm, prm, brick):
    """oracle.pm.Params matching a cube_params struct."""
    return pm.Params(n_fine=prm.n_fine, n_particles=prm.n_particles, ratio=prm.ratio, x_bytes=prm.x_bytes,
                     v_bytes=prm.v_bytes, box=prm.box, omega_m=prm.omega_m, omega_l=prm.omega_l,
                     deconv_power=prm.deconv_power, brick=brick)


def assert_store_equal(gpu, ref, what=""):
    """Integer parts bit-exact, v_c bit-exact (fixed-point mean)."""
    assert np.array_equal(gpu["counts"], ref.counts), f"{what}: counts differ"
    assert np.array_equal(gpu["offsets"][1:], np.cumsum(ref.counts)), f"{what}: offsets differ"
    assert np.array_equal(gpu["vc"], ref.vc), f"{what}: v_c differ (max {np.max(np.abs(gpu['vc'] - ref.vc))})"
    for name in ("chi", "nu"):
        g, r = gpu[name], getattr(ref, name)
        bad = np.count_nonzero(g != r)
        assert bad == 0, f"{what}: {bad} of {g.size} {name} codes differ"
    if gpu["ids"] is not None:
        assert np.array_equal(gpu["ids"], ref.ids), f"{what}: order (ids) differs"
