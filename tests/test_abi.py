"""C ABI checks that need no GPU: the library loads, exports every symbol
declared in include/simrank.h, and its host-only batch planner matches the
oracle's §8 partition."""
import os
import re

import numpy as np
import pytest

import paper_1711_00121_gb300 as P
from oracle import simrank_oracle as O
from synth import er_graph, batch_with_new_nodes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(simrank_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = P.lib()
    decl = declared_symbols()
    assert decl, "no declarations found"
    for name in sorted(decl):
        assert hasattr(L, name), name
    assert decl == set(P.SIGNATURES), decl ^ set(P.SIGNATURES)


def test_struct_layouts_match_header(tmp_path):
    """Size and field offsets of the ctypes structs equal the C compiler's
    layout of include/simrank.h (a small C program prints them)."""
    import ctypes
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"simrank_update": P.Update, "simrank_config": P.Config, "simrank_stats": P.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "simrank.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def _expand_oracle(ups, n_old):
    plus, minus = O.net_update(ups)
    dels, ins = O.partition_similar_sink(plus, minus, lambda x: x < n_old)
    out = [(j, -1, list(srcs)) for j, srcs in dels]
    exists = set(range(n_old))
    for j, srcs in ins:
        for _, part in O.block_case(srcs, j, lambda x: x in exists):
            out.append((j, 1, list(part)))
            exists.update(part)
            exists.add(j)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_plan_batch_matches_oracle_partition(seed):
    n = 40
    s, d = er_graph(n, 120, seed)
    ups, _ = batch_with_new_nodes(n, s, d, 60, seed, frac_new=0.3, reuse_target=0.5)
    # add cancelling pairs
    extra = []
    for t in range(5):
        i, j = int(ups[t][0]), int(ups[t][1])
        if ups[t][2] > 0:
            extra += [(i, j, -1), (i, j, 1)]
    allu = ups.tolist() + extra
    got = P.plan_batch(allu, n)
    want = _expand_oracle(allu, n)
    assert got == want


def test_plan_batch_rejects_bad_net_count():
    with pytest.raises(P.SimrankError):
        P.plan_batch([(0, 1, 1), (0, 1, 1)], 5)


def test_default_config_matches_header():
    """simrank_default_config is host only; its values are the ones the header
    documents."""
    from paper_1711_00121_gb300 import _binding as B

    cfg = B.default_config()
    assert cfg.C == 0.6 and cfg.K == 15 and cfg.s_precision == 32
    assert cfg.mode == P.MODE_DENSE and cfg.aff == 1 and cfg.relabel == 1
    assert cfg.upper_only == 1 and cfg.tc == 0 and cfg.defer == 0 and cfg.vec_fp64 == 0
    assert cfg.init_tol == 0.0 and cfg.init_max_sweeps == 400


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises; there is no CPU fallback."""
    import subprocess
    import sys

    code = (
        "import paper_1711_00121_gb300._binding as B\n"
        f"B.LIB_PATH = {str(tmp_path / 'missing.so')!r}\n"
        "B._lib = None\n"
        "try:\n"
        "    B.lib()\n"
        "except ImportError as e:\n"
        "    print('raised', e)\n"
        "else:\n"
        "    raise SystemExit('no error')\n"
    )
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    assert "raised" in r.stdout
