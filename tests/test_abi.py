"""Host-only checks of the C-ABI library: it builds, loads, and exports every
entry point that include/ephdc.h declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re

from paper_2511_00737_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ephdc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hdc_encode", "bfv_encode_plain", "bfv_ptct_similarity",
                     "bfv_decrypt_scores", "bfv_keygen", "bfv_encrypt_model", "ephdc_infer",
                     "ephdc_ctx_create", "ephdc_ctx_destroy", "ephdc_last_error"]:
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2511_00737_gb300 import ephdc
    assert set(declared_functions()) <= set(ephdc.exported_symbols())


def test_invalid_parameters_rejected_on_host():
    """Argument checks run before any device call."""
    from paper_2511_00737_gb300 import ephdc
    lib = ephdc.lib()
    for bad in [dict(n=1000), dict(L=1), dict(k=3, k_in=2), dict(r=3), dict(F=100),
                dict(hv_bits=9), dict(max_batch=0), dict(r=4096),
                dict(t=65539), dict(t=40961 * 3), dict(t=786433 * 2048 + 1),
                dict(prime_bits=31), dict(prime_bits=12), dict(scale_shift=31),
                dict(t=536903681, prime_bits=27)]:
        p = dict(n=4096, L=3, k=2, k_in=2, r=8, D=100, F=64, hv_bits=4, shift=3, max_batch=16,
                 sigma=3.2)
        p.update(bad)
        prm = ephdc.ephdc_params(**p)
        out = ctypes.c_void_p()
        st = lib.ephdc_ctx_create(ctypes.byref(prm), ctypes.byref(out))
        assert st == -1, bad
        assert not out.value
        assert lib.ephdc_last_error(None)
