"""Cool-chic overfitting on GB300 (sm_103a): one encoder iteration (forward, hand-written
backward, Adam) over every pixel of an image, as CUDA kernels behind a C ABI
(include/coolchic.h).

Modules:
  coolchic        ctypes binding of the C ABI (argument marshalling only)
  autograd        CoolChicIter, the iteration as a torch.autograd.Function
  batch           several images at once on separately loaded library copies; autotune
  build           nvcc build of the library for sm_103a, in-tree
  synthetic       seeded synthetic images and initial parameters (inputs only)
  warm_bench      the learned warm start against plain overfitting
  batch_bench, codec_bench, profile, trace
                  measurement tools
  eager_baseline  the same iteration in plain PyTorch eager operations, a comparison
                  baseline for bench.py; no library path calls it
"""
