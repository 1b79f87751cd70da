"""GB300-native chromatic Gibbs sampler for Gaussian Markov random fields (Brown, McMahan &
Self, arXiv 1702.05518).  The compute path is the CUDA library ``libgmrf.so`` (sm_103a) behind
the C ABI of ``include/gmrf.h``; ``paper_1702_05518_gb300.gmrf`` is its thin ctypes binding and
``paper_1702_05518_gb300.workloads`` generates seeded synthetic inputs."""
