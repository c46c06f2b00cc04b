"""GB300-native parallel reduction (Jradi, do Nascimento, Martins,
"A Fast and Generic GPU-Based Parallel Reduction Implementation").

The compute path is the C-ABI library ``libpr.so`` (hand-written sm_103a CUDA);
``paper_1710_07358_gb300.pr`` is its thin Python binding and
``paper_1710_07358_gb300.autograd`` wraps it in torch.autograd.Functions.
Loading the library is deferred to the first call, which raises if it was
not built: there is no fallback implementation.
"""
__all__ = ["pr", "synth", "metrics"]
