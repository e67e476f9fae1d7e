"""GB300-native LSB substitution steganography (embed / extract / changed
bytes) behind a C-ABI CUDA library; see ``include/stego.h``."""
