"""GB300-native DPD step loop (arxiv 1804.06205): CUDA engine behind a C ABI."""
