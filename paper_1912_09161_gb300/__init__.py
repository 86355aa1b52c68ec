"""GB300-native VELO reconstruction (LHCb Allen, paper section 2.3.1).

The reconstruction runs in the CUDA library built from ``csrc/`` (C ABI in
``include/velo.h``); ``velo`` is its ctypes binding.
"""
from .velo import (DeviceEvents, DeviceOutput, HostResult, Params, Reconstructor, VeloError, alloc_output,
                   load_library, suggested_caps, upload_events)

__all__ = ["DeviceEvents", "DeviceOutput", "HostResult", "Params", "Reconstructor", "VeloError", "alloc_output",
           "load_library", "suggested_caps", "upload_events"]
