"""GB300-native two-grid GMsFEM-preconditioned solver for mixed RT0/P0 Darcy flow.

The compute path is the C-ABI library ``libtgms`` (hand-written sm_103a CUDA,
``csrc/``); ``tgms`` is a thin ctypes binding with the same entry-point names.
``inputs`` holds the seeded synthetic input generators.  Importing the
package does not load the CUDA library; ``tgms.lib()`` does, and raises if it
has not been built.
"""
