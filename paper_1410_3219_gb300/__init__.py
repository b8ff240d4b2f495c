"""GB300-native moving Voronoi mesh hydrodynamics sweep (RICH scheme,
arXiv:1410.3219): a C-ABI CUDA library (librich.so) and its thin Python
binding.  Importing the package loads nothing; the binding loads the library
on first use and raises if it is missing."""
