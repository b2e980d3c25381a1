"""GB300-native periodic Ewald-RPY Brownian-dynamics step (Jain et al.).

The compute path is the CUDA library ``libbdgb.so`` (C ABI declared in
``include/bd.h``); :mod:`paper_1203_6208_gb300.binding` marshals arguments to
it.  :mod:`paper_1203_6208_gb300.inputs` draws the seeded synthetic systems.
"""
__all__ = ["inputs", "binding"]
