"""Region-segmented streaming pipelines on B300 (sm_103a).

The CUDA library (csrc/, built into librs.so) is reached through the ctypes
binding in `rs`; importing this package loads nothing until `rs` is used.
"""
