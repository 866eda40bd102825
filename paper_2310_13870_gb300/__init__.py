"""GB300 (sm_103a) implementation of the FastSimilarityGraph hot path.

``fsg``    -- Python binding of libfsg.so (include/fsg.h);
``inputs`` -- seeded synthetic workloads;
``build``  -- compiles libfsg.so in-tree with nvcc.

Importing the package loads nothing; ``fsg.load()`` loads the library.
"""
