"""The C ABI without a GPU: the library loads, exports every function include/*.h declares,
and rejects invalid parameter sets with CGEVAP_ERR_ARG and a message before touching a device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"^CGEVAP_API\s+[\w\s\*]+?\b(cgevap_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_14859_gb300 import build, binding
    build.build()
    return binding.lib()


def test_header_declares_functions():
    names = declared_functions()
    assert "cgevap_create" in names and "cgevap_step" in names
    assert len(names) >= 20


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_2412_14859_gb300 import binding
    assert set(declared_functions()) <= set(binding.all_signatures())


def _params(**kw):
    from paper_2412_14859_gb300 import binding
    base = dict(q=19, nx=8, ny=8, nz=8, rho_r_in=1.0, rho_b_in=1.0, tau_r=1.0, tau_b=1.0,
                sigma=0.0, beta=0.7, site_rule=1, threshold=0.5, sbar=3.0, storage=1)
    base.update(kw)
    p = binding.Params()
    for k, v in base.items():
        setattr(p, k, v)
    p.periodic = (ctypes.c_int * 3)(1, 1, 1)
    return p


@pytest.mark.parametrize("bad,needle", [
    (dict(q=7), "q must be"), (dict(q=9, nz=2), "D2Q9"), (dict(nx=0), "sizes"),
    (dict(tau_r=0.5), "tau"), (dict(tau_b=0.3), "tau"), (dict(beta=1.5), "beta"),
    (dict(rho_b_in=0.0), "densities"), (dict(sbar=0.0), "sbar"), (dict(site_rule=5), "rule"),
    (dict(storage=9), "storage"), (dict(nx=2048, ny=2048, nz=1024), "2^31"),
])
def test_invalid_params_rejected(lib, bad, needle):
    h = ctypes.c_void_p()
    rc = lib.cgevap_create(ctypes.byref(_params(**bad)), ctypes.byref(h))
    assert rc == -1
    assert needle in lib.cgevap_last_error(None).decode()
    assert not h.value


def test_null_handles_rejected(lib):
    assert lib.cgevap_step(None, 1) == -1
    assert lib.cgevap_set_outlets(None, 1.0, 1.0) == -1
    assert lib.cgevap_set_flux_heated(None, 1e-3, 0.5, 10.0, 1) == -1
    assert lib.cgevap_get_flux_field(None, None) == -1
    assert lib.cgevap_destroy(None) == 0
    assert lib.cgevap_bytes_per_update(None) == 0.0
    assert lib.cgevap_get_ledger_async(None, None) == -1


def test_ledger_record_decodes():
    """The 40-byte record cgevap_get_ledger_async copies is the public cgevap_ledger; the
    binding decodes it from a byte tensor."""
    import torch
    from paper_2412_14859_gb300.binding import Ledger, Sim
    assert ctypes.sizeof(Ledger) == 40
    rec = Ledger(evaporated=1.5, last_removed=0.25, site_steps=7, last_sites=3, steps=9)
    buf = torch.frombuffer(bytearray(bytes(rec) + bytes(8)), dtype=torch.uint8)
    assert Sim.ledger_from(buf) == {"evaporated": 1.5, "last_removed": 0.25, "site_steps": 7,
                                    "last_sites": 3, "steps": 9}
