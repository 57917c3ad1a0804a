"""GB300-native Wilson-Dirac conjugate gradient (sm_103a CUDA behind a C ABI)."""
