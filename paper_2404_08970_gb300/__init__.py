"""GB300-native fast Gromov-Wasserstein gradient (arXiv 2404.08970).

The compute path is the CUDA library libgw_fgc.so (see include/gw.h); this
package only builds it (build.py) and marshals arguments to it (_lib.py).
Importing the package does not load the library.
"""
