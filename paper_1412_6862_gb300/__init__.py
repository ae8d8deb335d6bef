"""GB300-native Hamming(n,k) decoder (sm_103a CUDA kernels behind a C ABI)."""
