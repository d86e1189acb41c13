"""FP64 oracle of the CT augmentation hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product library never calls it and
shares no code with it.  See ``oracle.c`` for the definitions and
``ref.py`` for the Python entry points.
"""
