"""The checked build (libdsasa_checked.so, compiled with DSASA_CHECKED): every data-dependent
index of the atom kernels into an array of atoms is verified on the device, a bad one setting
DSASA_ERR_CHECK.  On valid inputs it must report OK and give exactly the normal library's
results (the checks change no arithmetic)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


class _Cfg(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skin", ctypes.c_double), ("max_atoms", ctypes.c_int64),
                ("max_cells", ctypes.c_int64), ("carry", ctypes.c_int)]


@pytest.fixture(scope="module")
def checked():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_10462_gb300 import build
    L = ctypes.CDLL(build.build_checked())
    vp = ctypes.c_void_p
    L.dsasa_default_config.argtypes = [ctypes.POINTER(_Cfg)]
    L.dsasa_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(_Cfg)]
    L.dsasa_compute.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int64, vp, vp]
    L.dsasa_status_sync.argtypes = [vp]
    L.dsasa_destroy.argtypes = [vp]
    return torch, L


def _run_checked(torch, L, x, r, skin, steps):
    vp = ctypes.c_void_p
    cfg = _Cfg()
    L.dsasa_default_config(ctypes.byref(cfg))
    cfg.skin = skin
    cfg.carry = 2
    h = vp()
    assert L.dsasa_create(ctypes.byref(h), 0, vp(torch.cuda.current_stream().cuda_stream), ctypes.byref(cfg)) == 0
    out = []
    rt = torch.as_tensor(r, device="cuda")
    for xs in [x] + steps:
        xt = torch.as_tensor(xs, device="cuda")
        a = torch.empty(len(r), dtype=torch.float64, device="cuda")
        g = torch.empty((len(r), 3), dtype=torch.float64, device="cuda")
        assert L.dsasa_compute(h, vp(xt.data_ptr()), vp(rt.data_ptr()), 1.4, len(r), vp(a.data_ptr()),
                               vp(g.data_ptr())) == 0
        assert L.dsasa_status_sync(h) == 0          # no bounds check fired
        out.append((a.cpu().numpy(), g.cpu().numpy()))
    L.dsasa_destroy(h)
    return out


@pytest.mark.parametrize("case", ["globule5000", "rna1000", "shell3000", "globule8000-steps"])
def test_checked_build_matches_the_library(checked, gen, case):
    torch, L = checked
    from paper_2401_10462_gb300 import api
    steps = []
    if case.startswith("globule8000"):
        m = gen.make("globule", 8000, 1)
        rng = np.random.default_rng(4)
        steps = [m.coords + rng.normal(scale=0.01 * (k + 1), size=m.coords.shape) for k in range(2)]
        skin = 1.0
    elif case.startswith("globule"):
        m, skin = gen.globule(5000, 0), 0.0
    elif case.startswith("rna"):
        m, skin = gen.rna(1000, 1), 0.0
    else:
        m, skin = gen.shell(3000, 2, r_out=45.0, thickness=14.0, chain=100), 0.0
    got = _run_checked(torch, L, m.coords, m.radii, skin, steps)
    ctx = api.Context(skin=skin, carry=2)
    for (a, g), xs in zip(got, [m.coords] + steps):
        ra = torch.empty(m.n, dtype=torch.float64, device="cuda")
        rg = torch.empty((m.n, 3), dtype=torch.float64, device="cuda")
        ctx.compute(torch.as_tensor(xs, device="cuda"), torch.as_tensor(m.radii, device="cuda"), ra, rg)
        ctx.status_sync()
        assert np.array_equal(a, ra.cpu().numpy())
        assert np.array_equal(g, rg.cpu().numpy())
    ctx.close()
