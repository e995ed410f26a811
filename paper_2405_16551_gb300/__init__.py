"""GB300-native DE/rand/1/bin (arXiv 2405.16551): CUDA kernels behind a C ABI."""
