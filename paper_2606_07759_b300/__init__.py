"""B300-native synthetic interaction-matrix generation (SynIM's method, arxiv 2606.07759).

The compute path is libsynim.so (hand-written sm_103a CUDA behind the C ABI
of include/synim.h); this package only marshals arguments, with PyTorch for
device memory and streams.  ``workloads`` holds the seeded synthetic inputs.
"""
from .abi import SynimError  # noqa: F401


def __getattr__(name):
    if name == "SynIM":
        from .synim import SynIM
        return SynIM
    raise AttributeError(name)
