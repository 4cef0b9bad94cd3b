"""The in-tree build: every source file under csrc/ is compiled into the
library, and every local header a source includes is a dependency of every
object, so that editing a header rebuilds the objects that inline it; and
the host setup gives the same bits whatever the number of OpenMP threads."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2008_01541_b300")
SRC = os.path.join(PKG, "csrc")


def _build_module():
    spec = importlib.util.spec_from_file_location("pd_build", os.path.join(PKG, "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_source_is_compiled():
    b = _build_module()
    cu = sorted(f for f in os.listdir(SRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(SRC) if f.endswith(".cpp"))
    assert sorted(b.CU) == cu
    assert sorted(b.CPP) == cpp


def test_every_local_header_is_a_dependency():
    b = _build_module()
    included = set()
    for f in os.listdir(SRC):
        if f.endswith((".cu", ".cpp", ".h", ".cuh")):
            included |= set(re.findall(r'#include\s+"([^"]+)"', open(os.path.join(SRC, f)).read()))
    local = {h for h in included if os.path.exists(os.path.join(SRC, h))}
    assert local, "no local headers found"
    missing = sorted(local - set(b.HEADERS))
    assert not missing, missing
    # and nothing listed that does not exist
    assert all(os.path.exists(os.path.join(SRC, h)) for h in b.HEADERS)


def test_host_setup_is_deterministic_across_thread_counts():
    # the ordering, assembly and symbolic phases and the host factorisation
    # run OpenMP loops over rows, columns and fronts; each entry is computed
    # by one thread in a fixed order, so Sigma_0 must not depend on the count
    import subprocess
    import sys
    code = ("import sys, hashlib; sys.path.insert(0, %r); import scenes, paper_2008_01541_b300 as pd; "
            "s = scenes.small_elbow(h=1.5); S, _ = pd.host_schur(s.X, s.tets, s.region, s.dirichlet, s.mu, 1000.0, 0.03); "
            "print(hashlib.sha256(S.tobytes()).hexdigest())") % ROOT
    digests = set()
    for nt in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        digests.add(r.stdout.strip().splitlines()[-1])
    assert len(digests) == 1
