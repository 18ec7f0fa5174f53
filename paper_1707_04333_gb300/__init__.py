"""GB300-native charge-conserving relativistic FETD-PIC particle step (arXiv:1707.04333).

The compute path is the C-ABI library built from `csrc/` (sm_103a CUDA + C++
host setup); `fetdpic` is its thin ctypes binding.  Import it explicitly:

    from paper_1707_04333_gb300 import fetdpic
"""
