"""GB300-native flux-reconstruction residual and RK stage update (arXiv 2308.06605 hot path).

The compute path lives in the C-ABI library built from `csrc/` (header `include/fr.h`); `fr`
is its thin ctypes binding.  `inputs` holds the seeded synthetic workloads.  Importing the
package loads nothing compiled; `fr.load()` does, and fails loudly when the library is missing.
"""
