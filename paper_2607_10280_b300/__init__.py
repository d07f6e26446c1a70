"""B300-native MPS-ANO-VQC feature extraction (arxiv 2607.10280).

The CUDA library is loaded on first use (``paper_2607_10280_b300.api``); importing
the package alone needs neither a GPU nor the built library, so that the seeded
input generators in ``synth`` can be used by tests on any machine.
"""

__all__ = ["synth", "api"]
