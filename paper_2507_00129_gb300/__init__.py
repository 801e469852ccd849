"""GB300 Lyman-alpha pixel-pair library (arxiv 2507.00129 hot path).

``synth`` (input generator) imports without CUDA; the CUDA-backed API is
``paper_2507_00129_gb300.api``, which loads ``_build/liblya.so`` on first use.
"""
