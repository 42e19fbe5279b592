"""GB300-native density-fitted J/K build (3-centre integrals, Cholesky
whitening, J/K contractions) behind a C ABI.  Importing the package loads
nothing; ``paper_2404_09452_gb300.dfjk`` loads the CUDA library."""
