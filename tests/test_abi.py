"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-only entry points agree with the oracle.  No GPU needed."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mscd_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    return mscd.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol():
    from paper_1301_0955_gb300 import mscd

    assert set(declared_functions()) <= set(mscd.SIGNATURES)


def test_strerror_and_version(lib):
    from paper_1301_0955_gb300 import mscd

    assert lib.mscd_version() >= 100
    for rc in range(-14, 1):
        assert mscd.strerror(rc) != "unknown status"


def test_scales_match_oracle(lib, orc):
    from paper_1301_0955_gb300 import mscd

    for x in (1, 2, 8, 20, 32, 100):
        a = mscd.scales_logspaced(0.5, 1.0, x)
        rc, b = orc.scales_logspaced(0.5, 1.0, x)
        assert rc == 0
        assert np.allclose(a, b, rtol=1e-15, atol=0)
    with pytest.raises(mscd.MscdError):
        mscd.scales_logspaced(0.5, 1.0, 0)


def test_no_device_is_an_error(lib):
    """Without a GPU the context cannot be created: the path fails loudly."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1301_0955_gb300 import mscd

    with pytest.raises(mscd.MscdError) as e:
        mscd.Context(0)
    assert e.value.rc in (mscd.EDEVICE, mscd.EINVAL)
