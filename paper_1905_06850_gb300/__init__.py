"""GB300-native deep pipelined Conjugate Gradients, p(l)-CG (arXiv:1905.06850).

``paper_1905_06850_gb300.plcg`` is the Python binding of the C-ABI library
``libplcg.so`` (CUDA kernels for sm_103a); ``paper_1905_06850_gb300.workloads``
builds seeded synthetic inputs.  Importing the package imports neither.
"""
