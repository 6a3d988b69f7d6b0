"""Host-side checks of the C ABI: the library loads, exports every function
that include/*.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_06350_gb300 import build, recon
    build.build()
    return recon.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(recon_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_abi():
    from paper_1709_06350_gb300 import recon
    assert set(declared_functions()) <= set(recon.EXPORTS)


def test_status_strings(lib):
    assert lib.recon_status_string(0) == b"RECON_OK"
    assert lib.recon_status_string(2) == b"RECON_E_DOMAIN"


@pytest.mark.parametrize("N,ok", [(4, True), (6, True), (8, True), (96, True), (512, True),
                                  (3, False), (2, False), (34, False), (50, False)])
def test_size_rules(lib, N, ok):
    """N even >= 4 whose hierarchy ends at <= 16^3 (34 -> 17 odd: coarsest 34^3)."""
    assert (lib.recon_workspace_bytes(N, 0) > 0) == ok


def test_workspace_size_scales(lib):
    b64 = lib.recon_workspace_bytes(512, 0)
    bmx = lib.recon_workspace_bytes(512, 1)
    n = 512 ** 3
    assert 2 * 8 * n < b64 < 3 * 8 * n
    assert bmx > b64


def test_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.recon_create(7, 10.0, 0, ctypes.byref(h)) == 1
    assert b"even" in lib.recon_last_error(None)
    assert lib.recon_create(32, -1.0, 0, ctypes.byref(h)) == 1
    assert lib.recon_create(32, 10.0, 9, ctypes.byref(h)) == 1
    assert not h.value


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_1709_06350_gb300 import recon
    with pytest.raises(TypeError):
        recon._dev_ptr(torch.zeros(4))


def test_slab_layouts_rejected_before_launch():
    """Bad slab layouts come back RECON_E_INVALID without touching a GPU."""
    import ctypes
    from paper_1709_06350_gb300 import recon
    from paper_1709_06350_gb300 import build
    build.build()
    lib = recon.load()
    fake = ctypes.c_void_p(256)

    def lay(N, planes, first, lo, hi):
        return ctypes.byref(recon.recon_slab(N, planes, first, lo, hi))

    bad = [lay(7, 7, 0, 0, 7),          # odd N
           lay(2048, 2048, 0, 0, 2048),  # beyond the 32-bit offset range
           lay(16, 12, -2, 1, 11),       # sweep needs two halo planes each side
           lay(16, 12, -2, 2, 11),
           lay(16, 20, -2, 2, 18),       # a slab holding a plane twice
           lay(16, 8, 0, 4, 4)]          # no own planes
    for L in bad:
        assert lib.recon_slab_sweep(L, 1.0, 0, fake, fake, 0.0, fake, None) == 1
    assert lib.recon_slab_residual(lay(16, 8, 0, 0, 8), 1.0, fake, fake, 0.0, fake, None) == 1
    # restriction: the fine array must hold both sons of every own coarse plane
    assert lib.recon_slab_restrict(lay(16, 8, 0, 0, 8), fake, lay(8, 5, 0, 0, 5), fake, None) == 1
    # prolongation: the coarse array must hold the parents' neighbours
    assert lib.recon_slab_prolong_add(lay(8, 4, 0, 0, 4), fake, None, 1.0, lay(16, 8, 0, 0, 8), fake,
                                      None) == 1
    assert lib.recon_slab_defect_min(lay(16, 16, 0, 0, 16), fake, fake, 0.0, fake, None) == 1
    assert b"recon_slab" in lib.recon_last_error(None)
