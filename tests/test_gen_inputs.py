"""The seeded input generator gives the same bits on every machine: its result
may not depend on how many OpenMP threads build it (a system that differs in
the last bits sends the FP32 Krylov solver down another iteration path)."""
import hashlib
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CODE = r"""
import hashlib, sys
sys.path.insert(0, {root!r})
import gen
A, b = gen.make_system(256, 192, 20, 21, 22)
print(hashlib.sha256(A.tobytes()).hexdigest(), hashlib.sha256(b.tobytes()).hexdigest())
"""


def test_generator_is_independent_of_the_thread_count():
    import gen

    gen.build()  # compile once, outside the child processes
    digests = set()
    for threads in ("1", "3", "8"):
        out = subprocess.run([sys.executable, "-c", _CODE.format(root=ROOT)], capture_output=True, text=True,
                             env={**os.environ, "OMP_NUM_THREADS": threads}, timeout=300)
        assert out.returncode == 0, out.stderr
        digests.add(out.stdout.strip())
    assert len(digests) == 1, digests


def test_generator_is_seeded():
    import gen

    b1 = gen.make_rhs(64, 48, 10, 7)
    b2 = gen.make_rhs(64, 48, 10, 7)
    b3 = gen.make_rhs(64, 48, 10, 8)
    assert hashlib.sha256(b1.tobytes()).digest() == hashlib.sha256(b2.tobytes()).digest()
    assert not (b1 == b3).all()
