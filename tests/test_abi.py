"""The C-ABI library without a GPU: it loads, exports every symbol the
header declares, and its host-side validation rejects bad descriptions
before any device work."""
import os
import re

import numpy as np
import pytest

from paper_1310_6380_gb300 import binding as bs
from paper_1310_6380_gb300 import cells

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bandstructure.h")).read()
    return sorted(set(re.findall(r"\b(bs_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported():
    declared = _declared()
    assert set(declared) == set(bs.EXPORTED), declared
    for name in declared:
        assert hasattr(bs._lib, name), name


def test_header_compiles_as_c(tmp_path):
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text('#include "bandstructure.h"\nint main(void){bs_cell_desc d; (void)d; return 0;}\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def _desc_args(cell, M=2, precision=bs.BS_PREC_FP64):
    return (cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16), cell.lam.copy(),
            cell.mu.copy(), cell.rho.copy(), M, precision)


@pytest.mark.parametrize("mutate, needle", [
    (lambda a: a.__setitem__(6, 4), "2M+1"),                          # 2M+1 = 9 > P = 8
    (lambda a: a[4].__setitem__(0, -1.0), "mu"),                      # mu <= 0
    (lambda a: a[3].__setitem__(0, -2.0), "lam"),                     # lam + mu <= 0
    (lambda a: a[5].__setitem__(1, 0.0), "rho"),                      # rho <= 0
    (lambda a: a[3].__setitem__(1, np.nan), "finite"),                # NaN
    (lambda a: a[2].__setitem__((0, 0), 7), "phase"),                 # phase index >= nphase
    (lambda a: a.__setitem__(7, 5), "precision"),                     # unknown precision
    (lambda a: a.__setitem__(1, a[0]), "basis"),                      # h1 parallel to h2
])
def test_create_rejects_bad_descriptions(mutate, needle):
    cell = cells.circle_cell(8, 0.3)
    args = list(_desc_args(cell))
    mutate(args)
    with pytest.raises(bs.BSError) as ei:
        bs.bs_create_cell(*args)
    assert ei.value.code == bs.BS_EINVAL
    assert needle in str(ei.value)


def test_null_handles_are_rejected():
    with pytest.raises(bs.BSError) as ei:
        bs.bs_assemble(None)
    assert ei.value.code == bs.BS_EINVAL
    bs.bs_destroy_cell(None)        # a no-op by contract


def test_binding_rejects_wrong_dtypes():
    cell = cells.circle_cell(8, 0.3)
    args = list(_desc_args(cell))
    args[2] = args[2].astype(np.int32)
    with pytest.raises(TypeError):
        bs.bs_create_cell(*args)


def test_ibz_path_matches_library_contract():
    """The generator's path is uniform in arc length and closed at Gamma."""
    for lat in ("square", "hex"):
        h1, h2 = cells.square() if lat == "square" else cells.hexagonal()
        Q = cells.ibz_path(lat, 31, h1, h2)
        qm = 2 * np.pi * np.linalg.inv(np.array([h1, h2]))
        k = Q @ qm.T
        steps = np.linalg.norm(np.diff(k, axis=0), axis=1)
        # straight segments: equal steps except the two that turn a corner
        assert np.allclose(Q[0], 0) and np.allclose(Q[-1], 0)
        assert np.sum(np.abs(steps - np.median(steps)) > 1e-9) <= 2
