"""oracle/wall_blake_faxen.h is what oracle/gen_wall_blake_faxen.py derives
from the definition of the wall correction (Section 2.1.1: the Faxen
operators applied to the image part of Blake's Green's function).  The
header is regenerated here with sympy, compiled with mb_oracle.c, and its
wall blocks and one-sided fields compared with the committed oracle's.  The
comparison is numerical, so a different sympy version that formats the same
expressions differently still passes."""
import os
import shutil
import subprocess

import numpy as np

from oracle import gen_wall_blake_faxen as G
from oracle import oracle as O

ODIR = os.path.dirname(os.path.abspath(O.__file__))


def test_committed_wall_header_is_the_generated_one(tmp_path, monkeypatch):
    (tmp_path / "wall_blake_faxen.h").write_text(G.render())
    shutil.copy(os.path.join(ODIR, "mb_oracle.c"), tmp_path / "mb_oracle.c")
    so = str(tmp_path / "libregen.so")
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", str(tmp_path / "mb_oracle.c"),
                    "-o", so, "-lm"], check=True, capture_output=True)
    regen = O.load(so)
    rng = np.random.default_rng(12)
    pts = np.column_stack([rng.uniform(-3, 3, (60, 2)), rng.uniform(0.2, 4.0, 60)])
    pairs = [(pts[i], pts[j]) for i in range(0, 60, 2) for j in (i, i + 1)]
    committed = [(O.wall_block(x, y, 0.37), O.source_faxen_fields(x, y, 0.37)) for x, y in pairs]
    monkeypatch.setattr(O, "_lib", regen)
    for (x, y), (W, (img, free)) in zip(pairs, committed):
        scale = np.abs(W).max()
        np.testing.assert_allclose(O.wall_block(x, y, 0.37), W, rtol=0, atol=1e-13 * scale)
        i2, f2 = O.source_faxen_fields(x, y, 0.37)
        np.testing.assert_allclose(i2, img, rtol=0, atol=1e-13 * np.abs(img).max())
        np.testing.assert_allclose(f2, free, rtol=0, atol=1e-13 * np.abs(free).max())
