"""GB300-native (sm_103a) MetaCache-GPU hot path: minhash database build and
read classification as CUDA kernels behind a C ABI (include/mc.h).

`build()` compiles libmc.so in-tree; `paper_2106_08150_gb300.mc` is the thin
Python binding (it refuses to import without the compiled library)."""
from ._build import build  # noqa: F401
