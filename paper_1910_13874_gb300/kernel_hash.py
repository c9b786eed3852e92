"""Hash of the sweep kernel's device code, used to tell whether recorded ncu counters still apply."""
import hashlib
import os

_SWEEP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "sweep.cu")


def sweep_kernel_hash() -> str:
    text = open(_SWEEP).read()
    a = text.index("// [sweep-kernel-source-begin]")
    b = text.index("// [sweep-kernel-source-end]")
    return hashlib.sha256(text[a:b].encode()).hexdigest()[:16]
