"""GB300-native UGKS on a global adaptive velocity space (arXiv 2212.05645).

The compute path is the CUDA library ``libavs_gb300.so`` (sources in
``csrc/``), reached through the ctypes binding in :mod:`.avs`.  Importing the
package loads nothing; :func:`load` builds nothing either and raises when the
library is missing.
"""
__all__ = ["workloads", "avs"]
