"""GB300 (sm_103a) library for degree- and path-adjusted kNN-graph search.

Iwasaki & Miyazaki, "Optimization of Indexing Based on k-Nearest Neighbor Graph
for Proximity Search in High-dimensional Data" (arXiv 1810.07355).

Submodules:
  onng   the Python binding of the C ABI in include/onng.h (CUDA library)
  synth  seeded synthetic workloads shaped like the paper's datasets
  build  in-tree build of libonng.so

Importing the package loads nothing; ``onng.load()`` builds/loads the library.
"""
