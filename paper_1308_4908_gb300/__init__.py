"""GB300-native multi-sensor HDR reconstruction by noise-aware local polynomial approximation.

The compute path is the CUDA library `libhdrlpa.so` (sm_103a) behind the C ABI
declared in `include/hdr_lpa.h`; `paper_1308_4908_gb300.hdr` is its thin
ctypes binding and `paper_1308_4908_gb300.synth` the seeded input generator.
"""
__all__ = ["hdr", "synth"]
