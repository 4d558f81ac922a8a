"""GB300-native quaternion Dirac-Coulomb-Breit AO->MO integral transformation.

The compute path is libqdt.so (CUDA, sm_103a) behind the C ABI of
include/qdt.h; ``qdt`` is its thin Python binding and ``synth`` the seeded
input recipe.
"""
__all__ = ["qdt", "synth", "build"]
