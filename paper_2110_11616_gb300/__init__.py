"""GB300-native compressed geometric arrays (CGA) for point clouds.

The hot path (quantize/encode, radix sort, dedupe and CGA compaction, decode,
merge, orthogonal projection, exact nearest neighbour, and the batched and
served forms) runs in hand-written CUDA kernels for sm_103a behind the C-ABI
library ``libcga.so`` declared in ``include/cga.h``.  ``cga`` holds the thin
Python binding; ``synth`` the seeded synthetic inputs.
"""
