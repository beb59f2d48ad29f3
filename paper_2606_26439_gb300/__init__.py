"""GB300-native late-interaction MaxSim scoring (TileMaxSim, arxiv 2606.26439).

The compute path is the C-ABI CUDA library ``libtms.so`` (sources in
``csrc/``, declarations in ``include/tms.h``) built for sm_103a.  The Python
binding :mod:`paper_2606_26439_gb300.tms` only marshals arguments into it;
there is no CPU fallback.
"""
