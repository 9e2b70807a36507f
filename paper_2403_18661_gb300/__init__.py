"""GB300-native (sm_103a) Aframe detection hot path.

Import `paper_2403_18661_gb300.abi` for the C-ABI binding (it loads the
CUDA library and fails loudly when it is missing) and
`paper_2403_18661_gb300.inputs` for the seeded synthetic inputs.
"""
