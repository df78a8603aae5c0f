"""GB300-native round-based independent-set 2D anisotropic mesh adaptation.

The compute path is the CUDA library behind the C interface declared in
``include/pm.h``; ``paper_1505_04694_gb300.pm`` is its Python binding.
Importing the package does not load the library; ``pm`` does.
"""
