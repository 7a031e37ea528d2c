"""GB300-native Pruned Landmark Labeling (Akiba, Iwata, Yoshida, SIGMOD 2013).

The index build (bit-parallel BFS stage, batched pruned BFS with redundancy
cleanup) and the label-merge distance query run as hand-written sm_103a CUDA
kernels inside ``libpll.so`` behind the C ABI declared in ``include/pll.h``.
``pll`` is the thin ctypes binding; ``graphgen`` makes seeded synthetic inputs.
"""
