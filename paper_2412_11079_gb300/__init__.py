"""GB300-native MAP-UOT: the Sinkhorn iteration for entropy-regularised
unbalanced optimal transport on sm_103a, behind the C-ABI library ``libuot``."""
