"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer (host, no GPU): a copy
built with -fsanitize=address,undefined runs every entry point on small inputs -- brute force and
its gradient, tree build and export, Algorithm 1, the replay of Algorithm 2 and of its adjoint,
the enumerations, the learned proposal's network -- and must finish without a report."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, oracle as o
rng = np.random.default_rng(0)
for n in (1, 2, 9, 300):
    p = rng.random((n, 3)).astype(np.float32); w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    nv = rng.normal(size=(n, 3)).astype(np.float32)
    q = rng.uniform(-0.2, 1.2, (7, 3)).astype(np.float32)
    for kind in (o.COULOMB, o.WINDING, o.SMOOTHDIST, o.AFFINE):
        kw = dict(kind=kind, softening=1e-3, alpha=30.0, affine=(0.4, -0.3, 0.8))
        nrm = nv if kind == o.WINDING else None
        o.brute(p, w, q, normals=nrm, **kw); o.brute_grad(p, w, q, normals=nrm, **kw)
        for d, leaf in ((4, 1), (4, 3), (2, 1)):
            t = o.Tree(p, w, nrm, leaf_size=leaf, d=d)
            t.meta(); t.export(); t.bh(q, 2.0, **kw)
            if d == 4:
                t.replay(q, S=2, seed=3, return_abs_sum=True, **kw)
                t.replay_grad(q, S=1, seed=3, **kw)
                t.enumerate(q, **kw); t.enumerate_grad(q, **kw)
                wt = rng.normal(scale=0.3, size=o.MLP_NPARAM)
                t.enumerate_learned(q, wt, 0.1, near=1.0, **kw)
                e = t.export()
                for node in np.nonzero(e["nchild"])[0][:3]:
                    t.child_features(int(node), q[0], kind == o.WINDING)
off = np.array([0, 2, 7, 71]); x = rng.normal(size=(71, 6)); tg = rng.random(71)
o.mlp_loss_grad(rng.normal(size=o.MLP_NPARAM), x, tg, off); o.mlp_forward(rng.normal(size=o.MLP_NPARAM), x)
o.philox([1, 2, 3, 4], [5, 6])
print("sanitized oracle ok")
'''


def test_oracle_under_asan_and_ubsan(tmp_path):
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("no AddressSanitizer runtime for gcc here")
    lib = str(tmp_path / "liboracle_san.so")
    subprocess.run(["gcc", "-O1", "-g", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                    os.path.join(ROOT, "oracle", "sbh_oracle.c"), "-o", lib, "-lm"], check=True)
    env = dict(os.environ, SBHO_LIB=lib, LD_PRELOAD=libasan, OMP_NUM_THREADS="2",
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "sanitized oracle ok" in r.stdout, r.stderr[-3000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-3000:]
