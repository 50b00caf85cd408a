"""The C-ABI library loads on a machine without a GPU and exports every
function that include/thiim.h declares (no compute calls are made here)."""
import ctypes


def test_header_declares_the_boundary_calls():
    import paper_1510_05218_gb300 as p
    names = set(p.declared_symbols())
    for n in ("thiim_create", "thiim_set_coeffs", "thiim_set_fields", "thiim_iterate", "thiim_residual",
              "thiim_build_coeffs", "thiim_destroy", "thiim_strerror"):
        assert n in names, n


def test_library_exports_every_declared_symbol():
    import paper_1510_05218_gb300 as p
    from paper_1510_05218_gb300 import build
    build.build()
    lib = p.load_library()
    missing = [n for n in p.declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.thiim_version() >= 10000
    assert lib.thiim_strerror(0) == b"ok"
    assert b"alignment" in lib.thiim_strerror(-2) or b"misaligned" in lib.thiim_strerror(-2)


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    import paper_1510_05218_gb300 as p
    lib = p.load_library()
    h = ctypes.c_void_p()
    assert lib.thiim_create(ctypes.byref(h), 0, 4, 4, 0, 3, None) == -1
    assert lib.thiim_create(ctypes.byref(h), 4, 4, 4, 7, 3, None) == -1
    assert lib.thiim_create(ctypes.byref(h), 4, 4, 4, 0, 99, None) == -1
    assert lib.thiim_create(None, 4, 4, 4, 0, 3, None) == -1
    assert lib.thiim_iterate(None, 1) == -1
    assert lib.thiim_residual(None, None) == -1


def test_no_cpu_fallback_in_the_product_package():
    """The binding never imports the oracle: the product path has no CPU route."""
    import pathlib
    pkg = pathlib.Path(__file__).resolve().parents[1] / "paper_1510_05218_gb300"
    for f in pkg.rglob("*.py"):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text, f


def test_every_declared_call_has_a_python_binding():
    """The binding mirrors the ABI: each call declared in include/thiim.h is
    wrapped under the same name in paper_1510_05218_gb300.thiim."""
    import paper_1510_05218_gb300.thiim as T
    names = T.declared_symbols()
    missing = [n for n in names if not callable(getattr(T, n, None))]
    assert not missing, missing
