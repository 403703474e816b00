"""SSH (Sketch, Shingle & Hash) index and query path for DTW similarity search,
written for one GB300 GPU (sm_103a).

The compute path is the C-ABI CUDA library declared in include/ssh.h
(paper_1610_07328_gb300/csrc, built into _build/libssh_gb300.so); ``binding``
marshals numpy arrays and torch CUDA tensors into it. ``synth`` generates the
seeded synthetic inputs (random walks, ECG-like beat trains, perturbed queries).

Submodules are imported on demand; ``synth`` does not need the library, and
any call into ``binding`` loads the library and raises if it is absent.
"""
__all__ = ["binding", "synth", "build_ext", "build"]


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (no GPU needed) and return its path."""
    from . import build_ext
    return build_ext.build(force=force)
