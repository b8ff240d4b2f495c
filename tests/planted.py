"""Copies of the oracle with one planted mistake, compiled on the CPU for the
tests that show a pin catches that mistake.  The copy is made in a scratch
folder; the oracle in the tree is never touched."""
import os
import subprocess

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def build_planted(tmp_path, old, new, within="static void predict("):
    """Compile the oracle with the single occurrence of `old` inside the
    function that starts with `within` replaced by `new`; returns the .so."""
    src = open(os.path.join(ORACLE, "orc_hydro.c")).read()
    a = src.index(within)
    b = src.index("\n}\n", a)
    body = src[a:b]
    assert body.count(old) == 1, old
    src = src[:a] + body.replace(old, new) + src[b:]
    d = tmp_path / "orc"
    d.mkdir()
    (d / "orc_hydro.c").write_text(src)
    for f in ("orc_exact.c", "orc_delaunay.c", "orc.h"):
        (d / f).write_text(open(os.path.join(ORACLE, f)).read())
    so = str(d / "liborc_planted.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", so, str(d / "orc_exact.c"), str(d / "orc_delaunay.c"), str(d / "orc_hydro.c"),
                           "-lm"])
    return so
