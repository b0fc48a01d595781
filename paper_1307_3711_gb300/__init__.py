"""GB300-native hot path of the laser-cluster molecular-dynamics method of
Holkundkar, arXiv:1307.3711: softened O(N^2) Coulomb direct sum fused with the
dipole-approximation laser field and the relativistic Boris push, behind the
C-ABI library ``libmd.so``.

Importing the package loads nothing; ``paper_1307_3711_gb300.md`` loads the
CUDA library and raises if it is missing.
"""
