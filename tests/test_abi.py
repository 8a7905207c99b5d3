"""The C ABI library loads without a GPU, exports every function that
include/*.h declares, and its host-only pivot tables equal the oracle's
bit for bit (Sec. 3: Alg. 3.1, Alg. 3.2, reverse, modulus)."""
import glob
import os
import re

import numpy as np
import pytest

from oracle import pivots as P
from paper_1401_2720_gb300 import build_ext
from paper_1401_2720_gb300 import jsvd as J
from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return J.library()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(jsvd_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(J.EXPORTED) <= set(names)


@pytest.mark.parametrize("name", ["modulus", "R", "C", "rR", "rC"])
@pytest.mark.parametrize("nb", [2, 4, 6, 10, 12, 16, 18, 20, 22, 24, 40, 48, 64, 80, 96, 128, 512])
def test_pivot_tables_bit_exact(lib, name, nb):
    a = J.pivot_table(name, nb)
    b = P.to_array(P.strategy(name, nb))
    assert a.dtype == b.dtype and np.array_equal(a, b)


def test_pivot_table_rejects_bad_orders(lib):
    with pytest.raises(J.JsvdError):
        J.pivot_table("modulus", 7)
    with pytest.raises(J.JsvdError):
        J.pivot_table("rR", 26)        # base order 26 > 24: Alg. 3.1 not run


def test_status_strings(lib):
    for s in range(0, 7):
        assert lib.jsvd_status_string(s)


def _struct_fields(name):
    """Field names of a typedef'd struct in include/jsvd.h, in order."""
    text = open(os.path.join(ROOT, "include", "jsvd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    return [decl.split()[-1] for decl in body.split(";") if decl.strip()]


def test_option_and_info_layouts_match_the_header(lib):
    """The ctypes structures mirror jsvd_opts / jsvd_info field by field (a
    missing field would let the library write past the caller's buffer)."""
    assert [f for f, _ in J.Opts._fields_] == _struct_fields("jsvd_opts")
    assert [f for f, _ in J.Info._fields_] == _struct_fields("jsvd_info")


def test_default_options(lib):
    import ctypes

    o = J.Opts()
    lib.jsvd_default_opts(ctypes.byref(o))
    assert (o.b, o.strategy, o.inner_strategy, o.inner_sweeps, o.max_sweeps, o.precision, o.sort) == \
        (0, 3, -1, 1, 30, 0, 1)
    assert o.contraction == 1          # JSVD_CONTRACT_SPLIT: tensor-core contractions by default
    assert J.make_opts(contraction="fp64").contraction == 0
