"""GB300-native SPIDER sampling step (Ross et al., arXiv 2508.12117).

The compute lives in libspider.so (hand-written sm_103a kernels behind the C
ABI of include/spider.h); `binding` marshals arguments to it, `autograd` wraps
the travel-time kernel as a torch.autograd.Function and `synth` draws the
seeded synthetic catalogs used by tests and the benchmark."""
from . import binding  # noqa: F401
from .binding import (BF16, FP8, FP32, TT_HOMOGENEOUS, TT_LINEAR_GRADIENT, TT_MLP,  # noqa: F401
                      Context, Net, NetDevice, SpiderError, load_library, make_config,
                      spider_philox_words)
