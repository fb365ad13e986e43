"""GB300-native even/odd staggered Dirac operator and multi-shift CG.

Submodules (imported explicitly, nothing heavy is loaded here):

* ``inputs``  seeded synthetic lattices and sources (no method arithmetic);
* ``lqcd``    ctypes binding of the C-ABI library ``liblqcd.so``;
* ``build``   nvcc build of that library for sm_103a;
* ``serve``   Python front end of the continuous-batching solve server.
"""
__version__ = "0.1.0"
