"""GB300-native Next Event Backtracking pass (Jendersie, "Next Event Backtracking").

The compute path lives in the CUDA library ``libneb.so`` (sources in
``csrc/``, C-ABI declared in ``include/neb.h``); :mod:`.neb` is its thin
ctypes binding and :mod:`.scenes` holds the seeded synthetic inputs.
"""
