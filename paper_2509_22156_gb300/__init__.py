"""GB300-native hot path of the parallel-in-time sparse-grid combination
method (Griebel, Schweitzer, Troska, arXiv 2509.22156).

The compute path is libpit.so (hand-written CUDA for sm_103a) behind the C
ABI in include/pit.h; ``binding`` is its thin ctypes binding, ``workloads``
holds the seeded synthetic workloads, ``build`` compiles the library.
"""

__all__ = ["binding", "workloads", "build"]
