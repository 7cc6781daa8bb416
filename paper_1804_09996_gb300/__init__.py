"""GB300-native Link-and-Code search (Douze, Sablayrolles, Jegou, CVPR 2018).

* ``lc``       ctypes binding of liblc.so (C ABI in include/lc.h), same entry point names;
* ``build``    in-tree build of liblc.so for sm_103a;
* ``datagen``  seeded synthetic workloads (stand-ins for Deep1B / BIGANN).

Importing the package loads nothing; ``lc.lib()`` loads the library on first use and
raises if it is not built.
"""
