"""GB300-native Force2Vec epoch engine (arXiv:2009.10035).

``f2v``     -- Python binding of the CUDA library (include/f2v.h).
``graphs``  -- seeded synthetic graph generators (inputs only).
``build``   -- compiles the CUDA library for sm_103a.
"""
