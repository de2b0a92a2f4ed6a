"""GB300 (sm_103a) ensemble transfer-entropy hot path: max-norm kNN search, marginal range
counts and the KSG digamma sum over batches of trial-shuffled surrogates (Wollstadt et al.,
PLoS ONE 2014), behind a C ABI (``include/te_gb300.h``) with a thin ctypes binding (``te``)."""
from . import inputs  # noqa: F401  (seeded synthetic inputs; no method arithmetic)
