"""GB300-native engine for text analytics on grammar-compressed corpora."""
